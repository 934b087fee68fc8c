// walk.cu -- field at the active particles (STARFORGE methods paper, Sec. 2.2
// and 2.2.1) and its adjoint.
//
// Groups: the distinct active particles, in Morton order, are cut into runs
// of <= G targets: under every node holding more than G targets, its
// children holding 1..G are packed greedily in octant order; a leaf holding
// more than G is cut; the root forms one group if it holds <= G.
//
// One warp walks the tree for one group (persistent warps take groups from
// an atomic counter).  The walk is a stack of node-id ranges; each round pops
// up to 32 nodes (one per lane) and applies the opening rule, in exact
// integer arithmetic on the 2^21 grid (conservative form of Sec. 2.2's
// "open if L/r > Theta"):
//   accept node n  iff  (i)  sum_a gap(cell of com_n, group box)^2 >= ceil(4^(21-l)/Theta^2)
//                  and  (ii) sum_a gap(node box, group box)^2     >= max(hq_group, hq_node)
// (gap in whole cells between closed cell intervals; hq = ceil((h/cell)^2)):
// every target then sees the node at L/r <= Theta and lies outside the
// softening support of every member (Sec. 2.2.1), so the Newtonian
// multipole is the node's field.  Accepted nodes go to the P2M list, opened
// leaves to the P2P range queue, opened internal nodes push their child
// range.  Lists live in shared memory; every full tile of 32 entries is
// evaluated at once: each lane stages one source in shared memory, relative
// to the group centre in FP32 (integer half-cell centre differences are
// exact in FP32, plus the FP32 offset stored per node / particle), then
// every lane (one target each) loops over the tile reading broadcast
// shared-memory values.  Potentials are summed per tile in FP32 and
// accumulated in FP64.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>
#include <mutex>

#include "sfg_internal.cuh"

namespace sfg {

constexpr unsigned FULL = 0xffffffffu;
constexpr int WALK_WARPS = 4;  // warps per block
constexpr int WALK_MINB = 6;   // resident blocks per SM the register budget must allow
constexpr int STK = 224;       // shared-memory stack capacity (ranges) per warp
constexpr int GSTK = 4096;     // spill stack capacity per warp of the retry launch
constexpr int MODE_EVAL = 0, MODE_COUNT = 1, MODE_DUMP = 2, MODE_VJP = 3, MODE_EVAL64 = 4, MODE_LIST = 5,
              MODE_TIDAL = 6, // forward evaluation plus the tidal tensor (stored lists only)
              MODE_JERK = 7,  // forward evaluation plus the jerk (stored lists only)
              MODE_TSTEP = 8, // sink two-body timestep minima only (stored lists only)
              MODE_LIST1 = 9; // one-pass list walk: lists staged per warp, then copied to reserved space
// list sizes per group written by the counting walk: P2M nodes, softened P2P
// ranges and particles, Newtonian P2P ranges and particles
constexpr int NCNT = 5;

struct WarpSmem {
    int2 stack[STK];
    int p2m[64];
    int2 leafq[64];
    float4 tP[32];
    float4 tA[32]; // P2M: (Qxx, Qyy, Qxy, Qxz); P2P: (h, 1/h, j bits, sink flag)
    float tB[32];  // P2M: Qyz
    int tN[32];    // P2M: node id (adjoint)
    // all-FP64 evaluation: source (x, y, z, m) and P2M Q[6] / P2P (h, 1/h, j, sink)
    double dP[32][4];
    double dA[32][6];
};

struct WalkParams {
    const int4 *W0, *W1, *W2;
    const int32_t *nfirst, *ncount;
    const unsigned long long *Whq;
    const float4 *E0, *E1, *E2;
    const float4 *pw;
    const int4 *pc;
    const uint64_t *key;
    const double *pos_s, *soft_s, *mass_s;
    const uint8_t *sink_s;
    const double *nM, *ncom, *nQ;
    const Frame *frames;   // [C] per-cloud frames
    int npart;             // particles
    const int32_t *pcloud; // sorted rank -> cloud (NULL: one cloud)
    int nclouds;
    // with timing on: [C] latest item end per cloud, [C] = earliest warp start (ns)
    unsigned long long *ctime;
    unsigned long long T[SFG_LMAX + 1];
    int nn;
    const int2 *gtab;
    const int *d_ngroups;
    const int *tgt;
    float4 *res_a;
    double *res_phi;
    double *res64; // all-FP64 evaluation: [U][4] (a, phi), accumulated
    float *res_T;  // tidal mode: [U][8] = T without its isotropic part (xx yy zz xy xz yz), that part, -; summed
    float *res_J;        // jerk mode: [U][4] = j (x y z), -; summed
    unsigned *res_TS;    // timestep mode: [U][2] = min t_c^2, min (r^2 + eps^2)^{3/2} / (m_s + m_s') (float bits)
    const float4 *pv;    // jerk mode: particle velocities, sorted (FP32)
    const float4 *nV;    // jerk mode: node mass-weighted velocities (FP32 of the FP64 sums)
    // relative opening criterion (off when gps == NULL): |g_prev| per sorted rank, alpha, G
    const double *gps;
    double ralpha, rG;
    // one-pass list walk: per-warp staging (stg_cap_m P2M ids; stg_cap_r
    // softened, then stg_cap_r Newtonian ranges), the warps of the main
    // launch (the retry launch's warps follow them), the final buffers'
    // capacities, and the reservations: [0] P2M entries [1] ranges [2] 1 if
    // the final buffers were short [3] groups whose lists outgrew the
    // staging (listed in rlist; their space is reserved, a list-writing
    // walk of just those groups fills it) [4] [5] the largest P2M list and
    // range list (softened or Newtonian) of a group
    int *rlist;
    int *stg_m;
    int2 *stg_r;
    int stg_cap_m, stg_cap_r, stg_main_warps;
    long long lcap_m, lcap_r;
    unsigned long long *lbump;
    long long *lmo_w, *lro_w; // where each group's lists were placed (the lmo / lro arrays)
    unsigned long long *counters; // [0] p2p [1] p2m [2] overflowed groups [3] work [4] retry work
    int *ovf_list;
    int *status;
    int2 *gstack;
    // work items: group g is split into K_g items; item k of K evaluates
    // the tiles t = k (mod K) of the group's walk
    const int *ioff;
    const int2 *items;   // (group, k), heaviest first
    const int *kcnt;     // K_g
    const int *soff;     // first partial slot of a split group
    int *gdone;          // items finished per split group
    float4 *part_a;      // [slots][32]
    double *part_phi;    // [slots][32]
    // debug lists and costs: 3 ints per group (P2M nodes, P2P leaves, P2P particles)
    int *dbg_counts;
    const long long *dbg_off;
    int *dbg_m, *dbg_p;
    // stored lists: sizes (NCNT per group), first entries, P2M node ids, P2P ranges
    const int *lcnt;
    const long long *lmo, *lro;
    int *lm;
    int2 *lr;
    // the P2P ranges expanded to sorted particle ranks: first entry per group, entries
    const long long *lpo;
    const int *lp;
    // adjoint
    const float4 *cot; // per distinct target: (cot_a, cot_phi)
    double *gpart;     // [n][4] sorted: d_pos, d_mass
    double *gnode;     // [nn][10]: gM, gcom[3], gQ sym[6]
    float *gpart32;    // [n][4]: source-side sums of the chunked evaluation (added to gpart)
    float *gnode32;    // [nn][12]: gM, gcom[3], gQ[6], -, - (added to gnode)
};

// Target-lane state of one group.
// Lane layout: the group's T targets are padded to T' = 2^lb >= T; lane l
// serves target l mod T' and source slice l / T' of every tile (R = 32 / T'
// slices), so a small group still uses every lane; partial sums are reduced
// over the slices once per group.
struct Tgt {
    bool has;
    int r;
    float ox, oy, oz, h, hinv;
    bool sink;
    int cg[3];
    int tp, R, tl, slice;
    float s22;                  // half-cell size of the group's cloud (FP32)
    double x64[3], h64, hinv64; // all-FP64 evaluation only
    float vx, vy, vz; // jerk / timestep mode: the target's velocity
    float mt;         // timestep mode: the target's mass
    // relative criterion: alpha * min |g_prev| over the group, the cloud's root side, cell^2
    bool rel;
    double rel_ag, rel_L0, rel_cell2;
    float rel_agf, rel_GL0f, rel_cell2f; // FP32 roundings of alpha min|g|, G L0^2, cell^2
};

// Exact FP32 -> FP64 conversion of a normal or zero float (every result of
// the flush-to-zero FP32 arithmetic here), on the integer pipes; infinities
// and NaN take the hardware conversion, out of line so that no FP64
// conversion is issued on the common path.
__device__ __noinline__ double f64_of_special(float x) { return (double)x; }

__device__ __forceinline__ double f64_of(float x)
{
    const unsigned b = __float_as_uint(x), e = (b >> 23) & 0xffu;
    if (e == 255u) return f64_of_special(x);
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    if (e == 0u) return __longlong_as_double((long long)sign);
    return __longlong_as_double(
        (long long)(sign | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(b & 0x7fffffu) << 29)));
}

// ------------------------------------------------------------ kernels ----
// Softened kernel of support h at separation r (u = r/h < 1 here):
// a = K (x_j - x_i), phi = P per unit mass (M4 cubic spline, Sec. 2.2.1).
__device__ __forceinline__ void soft_KP(float r, float rinv, float h, float hinv, float &K, float &P)
{
    float u = r * hinv;
    if (u >= 1.f) {
        float ri2 = rinv * rinv;
        K = ri2 * rinv;
        P = -rinv;
        return;
    }
    float h3inv = hinv * hinv * hinv;
    float u2 = u * u;
    if (u < 0.5f) {
        K = h3inv * fmaf(u2, fmaf(32.f, u, -38.4f), 10.6666667f);
        P = hinv * fmaf(u2, fmaf(u2, fmaf(6.4f, u, -9.6f), 5.33333333f), -2.8f);
    } else {
        float uinv = h * rinv;
        float uinv3 = uinv * uinv * uinv;
        K = h3inv * (fmaf(u, fmaf(u, fmaf(-10.6666667f, u, 38.4f), -48.f), 21.3333333f) - 0.0666666667f * uinv3);
        P = hinv * (fmaf(u2, fmaf(u, fmaf(u, fmaf(-2.13333333f, u, 9.6f), -16.f), 10.6666667f), -3.2f) +
                    0.0666666667f * uinv);
    }
}

// Same kernel plus K'(r)/r (for the tidal tensor of the adjoint).
__device__ __forceinline__ void soft_KPR(float r, float rinv, float h, float hinv, float &K, float &P, float &R)
{
    float u = r * hinv;
    float ri2 = rinv * rinv;
    if (u >= 1.f) {
        K = ri2 * rinv;
        P = -rinv;
        R = -3.f * K * ri2;
        return;
    }
    float h2inv = hinv * hinv, h3inv = h2inv * hinv, h5inv = h3inv * h2inv;
    float u2 = u * u;
    if (u < 0.5f) {
        K = h3inv * fmaf(u2, fmaf(32.f, u, -38.4f), 10.6666667f);
        P = hinv * fmaf(u2, fmaf(u2, fmaf(6.4f, u, -9.6f), 5.33333333f), -2.8f);
        R = h5inv * fmaf(96.f, u, -76.8f);
    } else {
        float uinv = h * rinv;
        float uinv2 = uinv * uinv, uinv3 = uinv2 * uinv;
        K = h3inv * (fmaf(u, fmaf(u, fmaf(-10.6666667f, u, 38.4f), -48.f), 21.3333333f) - 0.0666666667f * uinv3);
        P = hinv * (fmaf(u2, fmaf(u, fmaf(u, fmaf(-2.13333333f, u, 9.6f), -16.f), 10.6666667f), -3.2f) +
                    0.0666666667f * uinv);
        R = h5inv * (fmaf(-32.f, u, 76.8f) - 48.f * uinv + 0.2f * uinv2 * uinv3);
    }
}

// Pair rule (Sec. 2.2.1): gas-gas averages the kernels of h_i and h_j; a pair
// with a sink uses one kernel of support max(h_i, h_j).  Returned as the two
// kernels to average: ha = max(h_i, h_j) and hb (= the smaller support for
// gas-gas, = ha when a sink is involved).  hh = source (h, 1/h, j, sink flag).
__device__ __forceinline__ void pair_supports(const Tgt &T, const float4 &hh, float &ha, float &hainv, float &hb,
                                              float &hbinv)
{
    bool sink = T.sink || hh.w != 0.f;
    bool tbig = T.h >= hh.x;
    ha = tbig ? T.h : hh.x;
    hainv = tbig ? T.hinv : hh.y;
    float lo = tbig ? hh.x : T.h, loinv = tbig ? hh.y : T.hinv;
    hb = sink ? ha : lo;
    hbinv = sink ? hainv : loinv;
}

// ------------------------------------------------------- forward tiles ----
// One P2M interaction: monopole a = M d / r^3, phi = -M / r, plus the
// quadrupole a_Q = -Q d / r^5 + 5/2 (d.Qd) d / r^7, phi_Q = -(d.Qd) / (2 r^5).
template <bool QUAD, class SM>
__device__ __forceinline__ void fwd_p2m_step(const SM &S, int k, const Tgt &T, float &ax, float &ay, float &az,
                                             float &pt)
{
    float4 p = S.tP[k];
    float dx = p.x - T.ox, dy = p.y - T.oy, dz = p.z - T.oz;
    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float rinv = rsqrtf(r2);
    float ri2 = rinv * rinv;
    float Mri3 = p.w * (ri2 * rinv);
    if (QUAD) {
        float4 q = S.tA[k];
        float qyz = S.tB[k];
        float qzz = -(q.x + q.y);
        float Qd0 = fmaf(q.x, dx, fmaf(q.z, dy, q.w * dz));
        float Qd1 = fmaf(q.z, dx, fmaf(q.y, dy, qyz * dz));
        float Qd2 = fmaf(q.w, dx, fmaf(qyz, dy, qzz * dz));
        float ri5 = rinv * ri2 * ri2;
        float t = fmaf(dx, Qd0, fmaf(dy, Qd1, dz * Qd2)) * ri5; // d.Qd / r^5
        float c = fmaf(t, 2.5f * ri2, Mri3);
        ax = fmaf(c, dx, fmaf(-ri5, Qd0, ax));
        ay = fmaf(c, dy, fmaf(-ri5, Qd1, ay));
        az = fmaf(c, dz, fmaf(-ri5, Qd2, az));
        pt = fmaf(-p.w, rinv, fmaf(-0.5f, t, pt));
    } else {
        ax = fmaf(Mri3, dx, ax);
        ay = fmaf(Mri3, dy, ay);
        az = fmaf(Mri3, dz, az);
        pt = fmaf(-p.w, rinv, pt);
    }
}

template <bool QUAD, class SM>
__device__ __forceinline__ void fwd_p2m(const SM &S, int cnt, const Tgt &T, float &ax, float &ay, float &az,
                                        double &phi)
{
    float pt = 0.f;
#pragma unroll 2
    for (int k = T.slice; k < cnt; k += T.R) fwd_p2m_step<QUAD>(S, k, T, ax, ay, az, pt);
    phi += (double)pt;
}

template <class SM>
__device__ __forceinline__ void fwd_p2p(const SM &S, int cnt, const Tgt &T, float &ax, float &ay, float &az,
                                        double &phi)
{
    float pt = 0.f;
#pragma unroll 2
    for (int k = T.slice; k < cnt; k += T.R) {
        float4 p = S.tP[k];
        float4 hh = S.tA[k];
        float dx = p.x - T.ox, dy = p.y - T.oy, dz = p.z - T.oz;
        float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        float m = (__float_as_int(hh.z) == T.r) ? 0.f : p.w;
        float hm = fmaxf(T.h, hh.x);
        float K, Pk;
        if (r2 < hm * hm) {
            float ha, hainv, hb, hbinv;
            pair_supports(T, hh, ha, hainv, hb, hbinv);
            float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
            float r = r2 * rinv;
            float K1, P1, K2, P2;
            soft_KP(r, rinv, ha, hainv, K1, P1);
            soft_KP(r, rinv, hb, hbinv, K2, P2);
            K = 0.5f * (K1 + K2);
            Pk = 0.5f * (P1 + P2);
        } else {
            float rinv = rsqrtf(r2); // r2 >= hm^2 > 0
            K = rinv * rinv * rinv;
            Pk = -rinv;
        }
        float mK = m * K;
        ax = fmaf(mK, dx, ax);
        ay = fmaf(mK, dy, ay);
        az = fmaf(mK, dz, az);
        pt = fmaf(m, Pk, pt);
    }
    phi += (double)pt;
}

// ------------------------------------------------------- adjoint tiles ----

// One P2M tile of the adjoint for a fixed slice width TP.  With d = com - x_i,
// q = d.Qd, cd = c.d (c, cf the target's cotangents), the derivative of
// L = c.a + cf phi with respect to d is
//   gd = (M/r^3 + 5/2 q/r^7) c - Q c / r^5 + (5 cd/r^7 - cf/r^5) Q d
//      + [M/r^3 (cf - 3 cd/r^2) + (5 c.Qd + q (5/2 cf - 35/2 cd/r^2)) / r^7] d
// (the source's centre of mass gets +gd, the target -gd); dL/dM = cd/r^3 -
// cf/r; dL/dQ_ab = (w_a d_b + w_b d_a)/2 with w = (5/2 cd/r^7 - cf/(2 r^5)) d
// - c/r^5 (the off-diagonal sums are kept doubled and halved once at the end).
template <bool QUAD, class SM>
__device__ __forceinline__ void vjp_p2m_tile(const WalkParams &P, const SM &S, int cnt, const Tgt &T, float c0,
                                             float c1, float c2, float cf, float &gx, float &gy, float &gz)
{
    const int TP = T.tp, base = T.slice * TP;
    const int nxt = (T.tl + 1) & (TP - 1);
    const float ncf = -cf, cf25 = 2.5f * cf;
    float acc[10];
#pragma unroll
    for (int q = 0; q < 10; q++) acc[q] = 0.f;
    for (int j = 0; j < TP; j++) {
        const int k = base + ((T.tl + j) & (TP - 1));
        if (T.has && k < cnt) {
            float4 p = S.tP[k];
            float dx = p.x - T.ox, dy = p.y - T.oy, dz = p.z - T.oz;
            float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            float rinv = rsqrtf(r2);
            float ri2 = rinv * rinv, ri3 = ri2 * rinv;
            float cd = fmaf(c0, dx, fmaf(c1, dy, c2 * dz));
            float Mri3 = p.w * ri3;
            acc[0] = fmaf(cd, ri3, fmaf(ncf, rinv, acc[0]));
            float gd0, gd1, gd2;
            if (QUAD) {
                float ri5 = ri3 * ri2, ri7 = ri5 * ri2;
                float4 qa = S.tA[k]; // Qxx Qyy Qxy Qxz
                float qyz = S.tB[k];
                float qzz = -(qa.x + qa.y);
                float Qd0 = fmaf(qa.x, dx, fmaf(qa.z, dy, qa.w * dz));
                float Qd1 = fmaf(qa.z, dx, fmaf(qa.y, dy, qyz * dz));
                float Qd2 = fmaf(qa.w, dx, fmaf(qyz, dy, qzz * dz));
                float Qc0 = fmaf(qa.x, c0, fmaf(qa.z, c1, qa.w * c2));
                float Qc1 = fmaf(qa.z, c0, fmaf(qa.y, c1, qyz * c2));
                float Qc2 = fmaf(qa.w, c0, fmaf(qyz, c1, qzz * c2));
                float q = fmaf(dx, Qd0, fmaf(dy, Qd1, dz * Qd2));
                float cQd = fmaf(c0, Qd0, fmaf(c1, Qd1, c2 * Qd2));
                float kc = fmaf(2.5f * q, ri7, Mri3);
                float kq = fmaf(5.f * cd, ri7, ncf * ri5);
                float kd = fmaf(ri7, fmaf(q, fmaf(-17.5f * cd, ri2, cf25), 5.f * cQd),
                                Mri3 * fmaf(-3.f * cd, ri2, cf));
                gd0 = fmaf(kc, c0, fmaf(-ri5, Qc0, fmaf(kq, Qd0, kd * dx)));
                gd1 = fmaf(kc, c1, fmaf(-ri5, Qc1, fmaf(kq, Qd1, kd * dy)));
                gd2 = fmaf(kc, c2, fmaf(-ri5, Qc2, fmaf(kq, Qd2, kd * dz)));
                float sQ = 0.5f * kq;
                float w0 = fmaf(sQ, dx, -ri5 * c0), w1 = fmaf(sQ, dy, -ri5 * c1), w2 = fmaf(sQ, dz, -ri5 * c2);
                acc[4] = fmaf(w0, dx, acc[4]);
                acc[5] = fmaf(w1, dy, acc[5]);
                acc[6] = fmaf(w2, dz, acc[6]);
                acc[7] = fmaf(w0, dy, fmaf(w1, dx, acc[7]));
                acc[8] = fmaf(w0, dz, fmaf(w2, dx, acc[8]));
                acc[9] = fmaf(w1, dz, fmaf(w2, dy, acc[9]));
            } else {
                // monopole: a = M d / r^3, phi = -M / r
                float kd = Mri3 * fmaf(-3.f * cd, ri2, cf);
                gd0 = fmaf(Mri3, c0, kd * dx);
                gd1 = fmaf(Mri3, c1, kd * dy);
                gd2 = fmaf(Mri3, c2, kd * dz);
            }
            acc[1] += gd0;
            acc[2] += gd1;
            acc[3] += gd2;
            gx -= gd0;
            gy -= gd1;
            gz -= gd2;
        }
#pragma unroll
        for (int q = 0; q < (QUAD ? 10 : 4); q++) acc[q] = __shfl_sync(FULL, acc[q], nxt, TP);
    }
    if (QUAD) {
        acc[7] *= 0.5f;
        acc[8] *= 0.5f;
        acc[9] *= 0.5f;
    }
    const int k = base + T.tl;
    if (k < cnt && S.tN[k] >= 0) {
        double *dst = P.gnode + 10 * (size_t)S.tN[k];
#pragma unroll
        for (int q = 0; q < (QUAD ? 10 : 4); q++)
            if (acc[q] != 0.f) atomicAdd(dst + q, (double)acc[q]);
    }
}

// Target side accumulates -dL/dd in registers.  Source side: within each
// slice of T' lanes, step j pairs lane t with source (t + j) mod T' of the
// slice's block of T' sources, and every lane hands its running source
// accumulator to lane t - 1 after each step; after T' steps lane t holds the
// complete sum (over the group's targets) for source t of the block and adds
// it to that source's gradient.
template <bool QUAD, class SM>
__device__ __forceinline__ void vjp_p2m(const WalkParams &P, const SM &S, int cnt, const Tgt &T, float c0,
                                        float c1, float c2, float cf, float &gx, float &gy, float &gz, int lane)
{
    vjp_p2m_tile<QUAD>(P, S, cnt, T, c0, c1, c2, cf, gx, gy, gz);
}

template <class SM>
__device__ __forceinline__ void vjp_p2p(const WalkParams &P, const SM &S, int cnt, const Tgt &T, float c0,
                                        float c1, float c2, float cf, float &gx, float &gy, float &gz, int lane)
{
    const int tp = T.tp, base = T.slice * tp;
    const int nxt = (T.tl + 1) & (tp - 1);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, am = 0.f;
    for (int jj = 0; jj < tp; jj++) {
        const int k = base + ((T.tl + jj) & (tp - 1));
        if (T.has && k < cnt) {
            float4 p = S.tP[k];
            float4 hh = S.tA[k];
            int j = __float_as_int(hh.z);
            if (j != T.r) {
                float dx = p.x - T.ox, dy = p.y - T.oy, dz = p.z - T.oz;
                float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                float ha, hainv, hb, hbinv;
                pair_supports(T, hh, ha, hainv, hb, hbinv);
                float hm = ha;
                float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
                float K, Pp, R;
                if (r2 < hm * hm) {
                    float r = r2 * rinv;
                    float K1, P1, R1, K2, P2, R2;
                    soft_KPR(r, rinv, ha, hainv, K1, P1, R1);
                    soft_KPR(r, rinv, hb, hbinv, K2, P2, R2);
                    K = 0.5f * (K1 + K2);
                    Pp = 0.5f * (P1 + P2);
                    R = 0.5f * (R1 + R2);
                } else {
                    float ri2 = rinv * rinv;
                    K = ri2 * rinv;
                    Pp = -rinv;
                    R = -3.f * K * ri2;
                }
                float m = p.w;
                float cd = fmaf(c0, dx, fmaf(c1, dy, c2 * dz));
                float mK = m * K;
                float sv = m * fmaf(R, cd, cf * K);
                float l0 = fmaf(mK, c0, sv * dx);
                float l1 = fmaf(mK, c1, sv * dy);
                float l2 = fmaf(mK, c2, sv * dz);
                a0 += l0;
                a1 += l1;
                a2 += l2;
                am += fmaf(K, cd, Pp * cf);
                gx -= l0;
                gy -= l1;
                gz -= l2;
            }
        }
        a0 = __shfl_sync(FULL, a0, nxt, tp);
        a1 = __shfl_sync(FULL, a1, nxt, tp);
        a2 = __shfl_sync(FULL, a2, nxt, tp);
        am = __shfl_sync(FULL, am, nxt, tp);
    }
    const int k = base + T.tl;
    if (k < cnt && __float_as_int(S.tA[k].z) >= 0) {
        double *dst = P.gpart + 4 * (size_t)__float_as_int(S.tA[k].z);
        if (a0 != 0.f) atomicAdd(dst, (double)a0);
        if (a1 != 0.f) atomicAdd(dst + 1, (double)a1);
        if (a2 != 0.f) atomicAdd(dst + 2, (double)a2);
        if (am != 0.f) atomicAdd(dst + 3, (double)am);
    }
}

// ------------------------------------------------- all-FP64 evaluation ----
__device__ __forceinline__ void soft_KP64(double r, double rinv, double h, double hinv, double &K, double &P)
{
    double u = r * hinv;
    if (u >= 1.0) {
        K = rinv * rinv * rinv;
        P = -rinv;
        return;
    }
    double h3inv = hinv * hinv * hinv, u2 = u * u;
    if (u < 0.5) {
        K = h3inv * (32.0 / 3.0 + u2 * (-192.0 / 5.0 + 32.0 * u));
        P = hinv * (-14.0 / 5.0 + u2 * (16.0 / 3.0 + u2 * (-48.0 / 5.0 + 32.0 / 5.0 * u)));
    } else {
        double uinv = h * rinv;
        K = h3inv * (64.0 / 3.0 + u * (-48.0 + u * (192.0 / 5.0 - 32.0 / 3.0 * u)) - uinv * uinv * uinv / 15.0);
        P = hinv * (uinv / 15.0 + u2 * (32.0 / 3.0 + u * (-16.0 + u * (48.0 / 5.0 - 32.0 / 15.0 * u))) - 16.0 / 5.0);
    }
}

template <bool QUAD>
__device__ __forceinline__ void stage_p2m64(const WalkParams &P, WarpSmem &S, const int *list, int cnt, int lane)
{
    if (lane < cnt) {
        int id = list[lane];
        for (int a = 0; a < 3; a++) S.dP[lane][a] = P.ncom[3 * (size_t)id + a];
        S.dP[lane][3] = P.nM[id];
        if (QUAD)
            for (int q = 0; q < 6; q++) S.dA[lane][q] = P.nQ[6 * (size_t)id + q];
    }
    __syncwarp();
}

__device__ __forceinline__ void stage_p2p64(const WalkParams &P, WarpSmem &S, int cnt, int &qh, int &qoff, int lane)
{
    int j = -1, filled = 0;
    for (int it = 0; filled < cnt && it < 66; it++) {
        int2 hr = S.leafq[qh & 63];
        int take = min(hr.y - qoff, cnt - filled);
        if (take < 0) take = 0;
        if (lane >= filled && lane < filled + take) j = hr.x + qoff + (lane - filled);
        filled += take;
        qoff += take;
        if (qoff >= hr.y) {
            qh++;
            qoff = 0;
        }
    }
    if (filled < cnt) {
        if (lane == 0) atomicOr(P.status, ST_ETIMEOUT);
        if (lane >= filled) j = -1;
    }
    if (lane < cnt && j >= 0) {
        for (int a = 0; a < 3; a++) S.dP[lane][a] = P.pos_s[3 * (size_t)j + a];
        S.dP[lane][3] = P.mass_s[j];
        double h = P.soft_s[j];
        S.dA[lane][0] = h;
        S.dA[lane][1] = 1.0 / h;
        S.dA[lane][2] = (double)j;
        S.dA[lane][3] = P.sink_s[j] ? 1.0 : 0.0;
    }
    __syncwarp();
}

template <bool QUAD>
__device__ __forceinline__ void fwd_p2m64(const WarpSmem &S, int cnt, const Tgt &T, double &ax, double &ay,
                                          double &az, double &phi)
{
    for (int k = T.slice; k < cnt; k += T.R) {
        double dx = S.dP[k][0] - T.x64[0], dy = S.dP[k][1] - T.x64[1], dz = S.dP[k][2] - T.x64[2];
        double M = S.dP[k][3];
        double r2 = dx * dx + dy * dy + dz * dz;
        double rinv = 1.0 / sqrt(r2);
        double ri3 = rinv * rinv * rinv;
        ax += M * dx * ri3;
        ay += M * dy * ri3;
        az += M * dz * ri3;
        phi -= M * rinv;
        if (QUAD) {
            const double *Q = S.dA[k]; // xx yy zz xy xz yz
            double Qd0 = Q[0] * dx + Q[3] * dy + Q[4] * dz;
            double Qd1 = Q[3] * dx + Q[1] * dy + Q[5] * dz;
            double Qd2 = Q[4] * dx + Q[5] * dy + Q[2] * dz;
            double dQd = dx * Qd0 + dy * Qd1 + dz * Qd2;
            double ri5 = ri3 * rinv * rinv, ri7 = ri5 * rinv * rinv;
            ax += -Qd0 * ri5 + 2.5 * dQd * dx * ri7;
            ay += -Qd1 * ri5 + 2.5 * dQd * dy * ri7;
            az += -Qd2 * ri5 + 2.5 * dQd * dz * ri7;
            phi += -0.5 * dQd * ri5;
        }
    }
}

__device__ __forceinline__ void fwd_p2p64(const WarpSmem &S, int cnt, const Tgt &T, double &ax, double &ay,
                                          double &az, double &phi)
{
    for (int k = T.slice; k < cnt; k += T.R) {
        int j = (int)S.dA[k][2];
        if (j == T.r) continue;
        double dx = S.dP[k][0] - T.x64[0], dy = S.dP[k][1] - T.x64[1], dz = S.dP[k][2] - T.x64[2];
        double m = S.dP[k][3];
        double r2 = dx * dx + dy * dy + dz * dz;
        double hj = S.dA[k][0], hjinv = S.dA[k][1];
        bool sink = T.sink || S.dA[k][3] != 0.0;
        bool tbig = T.h64 >= hj;
        double ha = tbig ? T.h64 : hj, hainv = tbig ? T.hinv64 : hjinv;
        double lo = tbig ? hj : T.h64, loinv = tbig ? hjinv : T.hinv64;
        double hb = sink ? ha : lo, hbinv = sink ? hainv : loinv;
        double rinv = r2 > 0.0 ? 1.0 / sqrt(r2) : 0.0;
        double K, Pk;
        if (r2 < ha * ha) {
            double r = r2 * rinv, K1, P1, K2, P2;
            soft_KP64(r, rinv, ha, hainv, K1, P1);
            soft_KP64(r, rinv, hb, hbinv, K2, P2);
            K = 0.5 * (K1 + K2);
            Pk = 0.5 * (P1 + P2);
        } else {
            K = rinv * rinv * rinv;
            Pk = -rinv;
        }
        ax += m * K * dx;
        ay += m * K * dy;
        az += m * K * dz;
        phi += m * Pk;
    }
}

// --------------------------------------------------------- tile staging ----
template <bool QUAD, bool NODEID, class SM>
__device__ __forceinline__ void stage_p2m(const WalkParams &P, SM &S, const int *list, int cnt, const Tgt &T,
                                          int lane)
{
    if (lane < cnt) {
        int id = list[lane];
        if ((unsigned)id < (unsigned)P.nn) {
            float4 e0 = P.E0[id];
            float4 e2 = P.E2[id];
            float px = fmaf((float)(__float_as_int(e2.y) - T.cg[0]), T.s22, e0.x);
            float py = fmaf((float)(__float_as_int(e2.z) - T.cg[1]), T.s22, e0.y);
            float pz = fmaf((float)(__float_as_int(e2.w) - T.cg[2]), T.s22, e0.z);
            S.tP[lane] = make_float4(px, py, pz, e0.w);
            if (QUAD) {
                S.tA[lane] = P.E1[id];
                S.tB[lane] = e2.x;
            }
        } else { // not a node (a corrupt list): massless and far, no gradient
            atomicOr(P.status, ST_ETIMEOUT);
            id = -1;
            S.tP[lane] = make_float4(3e18f, 0.f, 0.f, 0.f);
            if (QUAD) {
                S.tA[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
                S.tB[lane] = 0.f;
            }
        }
        if (NODEID) S.tN[lane] = id;
    }
    __syncwarp();
}

template <class SM>
__device__ __forceinline__ void stage_p2p(const WalkParams &P, SM &S, int cnt, int &qh, int &qoff, const Tgt &T,
                                          int lane)
{
    int j = -1, filled = 0;
    // at most 64 queued ranges can be pending; each iteration consumes one
    // range or completes the tile
    for (int it = 0; filled < cnt && it < 66; it++) {
        int2 hr = S.leafq[qh & 63];
        int take = min(hr.y - qoff, cnt - filled);
        if (take < 0) take = 0;
        if (lane >= filled && lane < filled + take) j = hr.x + qoff + (lane - filled);
        filled += take;
        qoff += take;
        if (qoff >= hr.y) {
            qh++;
            qoff = 0;
        }
    }
    if (filled < cnt) {
        if (lane == 0) atomicOr(P.status, ST_ETIMEOUT);
        if (lane >= filled) j = -1;
    }
    if (lane < cnt) {
        if (j >= 0 && j < P.npart) {
            float4 a = P.pw[j];
            int4 b = P.pc[j];
            float px = fmaf((float)(b.x - T.cg[0]), T.s22, a.x);
            float py = fmaf((float)(b.y - T.cg[1]), T.s22, a.y);
            float pz = fmaf((float)(b.z - T.cg[2]), T.s22, a.z);
            S.tP[lane] = make_float4(px, py, pz, a.w);
            float h = __int_as_float(b.w); // negative for a sink
            float ha = fabsf(h);
            S.tA[lane] = make_float4(ha, 1.f / ha, __int_as_float(j), h < 0.f ? 1.f : 0.f);
            S.tB[lane] = ha * ha;
        } else { // the ring ran dry or a corrupt range: massless and far, no gradient
            atomicOr(P.status, ST_ETIMEOUT);
            S.tP[lane] = make_float4(3e18f, 0.f, 0.f, 0.f);
            S.tA[lane] = make_float4(1.f, 1.f, __int_as_float(-1), 0.f);
            S.tB[lane] = 0.f;
        }
    }
    __syncwarp();
}

// ----------------------------------------------------------- the walk ----
// Opening rule for one node against the group box (see the file header):
// acc = accept (P2M); lf = sum its particle range pair by pair (P2P: an opened
// leaf, or an internal node wholly inside the group's softening reach, whose
// leaves would all be opened); op = open (push its children).  link/cnt:
// child range (op) or particle range (lf).
__device__ __forceinline__ void test_node(const WalkParams &P, const Tgt &T, int node, const int glo[3],
                                          const int ghi[3], unsigned long long hq, bool &acc, bool &lf, bool &op,
                                          bool &nw, int &link, int &cnt)
{
    acc = lf = op = nw = false;
    link = cnt = 0;
    if (node < 0) return;
    int4 w0 = P.W0[node], w1 = P.W1[node], w2 = P.W2[node];
    unsigned long long nhq = P.Whq[node];
    int level = w0.w & 255;
    bool leaf = (w0.w >> 8) & 1;
    int gc0 = max(0, max(glo[0] - w2.x - 1, w2.x - ghi[0] - 1));
    int gc1 = max(0, max(glo[1] - w2.y - 1, w2.y - ghi[1] - 1));
    int gc2 = max(0, max(glo[2] - w2.z - 1, w2.z - ghi[2] - 1));
    int gb0 = max(0, max(glo[0] - w1.x - 1, w0.x - ghi[0] - 1));
    int gb1 = max(0, max(glo[1] - w1.y - 1, w0.y - ghi[1] - 1));
    int gb2 = max(0, max(glo[2] - w1.z - 1, w0.z - ghi[2] - 1));
    unsigned long long sc = (unsigned long long)gc0 * (unsigned)gc0 + (unsigned long long)gc1 * (unsigned)gc1 +
                            (unsigned long long)gc2 * (unsigned)gc2;
    unsigned long long sb = (unsigned long long)gb0 * (unsigned)gb0 + (unsigned long long)gb1 * (unsigned)gb1 +
                            (unsigned long long)gb2 * (unsigned)gb2;
    unsigned long long need = nhq > hq ? nhq : hq;
    acc = sc >= P.T[level] && sb >= need;
    if (acc && T.rel) {
        // relative criterion (Sec. 2.2, from GADGET-2), conservative for every
        // target: G M L^2 <= alpha min|g_prev| (sc cell^2)^2, decided as the
        // oracle's IEEE FP64 products in the same order.  An FP32 screen goes
        // first: both of its sides lie within 16 FP32 roundings (< 2^-19
        // relative) of the FP64 sides, so where they differ by more than
        // 2^-18 and both are normal (no flush to zero, no overflow) it takes
        // the same decision; only the rest pays the FP64 products.
        const float Mf = __ldg(reinterpret_cast<const float *>(P.E0) + 4 * (size_t)node + 3);
        const float lhsf = Mf * (T.rel_GL0f * __int_as_float((127 - 2 * level) << 23));
        const float r2f = __ull2float_rn(sc) * T.rel_cell2f;
        const float rhsf = T.rel_agf * (r2f * r2f);
        const float lo_ok = 0x1p-100f, hi_ok = 0x1p100f;
        const bool normal = lhsf >= lo_ok && lhsf <= hi_ok && rhsf >= lo_ok && rhsf <= hi_ok;
        if (normal && lhsf <= rhsf * (1.f - 0x1p-18f)) {
            acc = true;
        } else if (normal && lhsf >= rhsf * (1.f + 0x1p-18f)) {
            acc = false;
        } else {
            const double L = ldexp(T.rel_L0, -level);
            const double lhs = __dmul_rn(__dmul_rn(P.rG, P.nM[node]), __dmul_rn(L, L));
            const double r2 = __dmul_rn((double)sc, T.rel_cell2);
            acc = lhs <= __dmul_rn(T.rel_ag, __dmul_rn(r2, r2));
        }
    }
    lf = !acc && leaf;
    op = !acc && !leaf;
    // an opened leaf that passes clause (ii): every pair it contributes is
    // beyond both softening supports (Newtonian)
    nw = lf && sb >= need;
    link = w1.w;
    cnt = w2.w;
    if (op) {
        // If even the farthest cell of the node lies inside the group's
        // softening reach, no descendant can pass clause (ii): every particle
        // below goes to the P2P list, so take the node's particle range at once.
        int f0 = max(0, max(w1.x - ghi[0] - 1, glo[0] - w0.x - 1));
        int f1 = max(0, max(w1.y - ghi[1] - 1, glo[1] - w0.y - 1));
        int f2 = max(0, max(w1.z - ghi[2] - 1, glo[2] - w0.z - 1));
        unsigned long long sf = (unsigned long long)f0 * (unsigned)f0 + (unsigned long long)f1 * (unsigned)f1 +
                                (unsigned long long)f2 * (unsigned)f2;
        if (sf < hq) {
            op = false;
            lf = true;
            link = P.nfirst[node];
            cnt = P.ncount[node];
        }
    }
}

// Walk state of one warp for one group.
struct WalkState {
    int sp, nm, qh, qt, qoff, qn, tile;
    int tot_m, tot_p, tot_leaf, tot_ln, tot_pn; // tot_ln / tot_pn: the Newtonian part of tot_leaf / tot_p
    long long off_s, off_n;                     // stored-list cursors of the softened / Newtonian ranges
    long long lim_m, lim_s, lim_n;              // ends of the group's stored-list regions
    float ax, ay, az;
    double phi;
    double dax, day, daz;
    float c0, c1, c2, cf;
    long long off_m, off_p;
    int *sm;      // one-pass list walk: this warp's staging
    int2 *ss, *sn;
};

// Append accepted nodes (acc) and P2P ranges (lf) of this round to the lists.
template <int MODE>
__device__ __forceinline__ void append_lists(const WalkParams &P, WarpSmem &S, WalkState &W, int node, bool acc,
                                             bool lf, bool nw, int link, int cnt, unsigned lt)
{
    unsigned ba = __ballot_sync(FULL, acc);
    unsigned bl = __ballot_sync(FULL, lf);
    int lc = __reduce_add_sync(FULL, lf ? cnt : 0);
    W.tot_m += __popc(ba);
    W.tot_leaf += __popc(bl);
    W.tot_p += lc;
    if (MODE == MODE_COUNT || MODE == MODE_LIST || MODE == MODE_LIST1) {
        unsigned bn = __ballot_sync(FULL, nw);
        W.tot_ln += __popc(bn);
        W.tot_pn += __reduce_add_sync(FULL, nw ? cnt : 0);
        if (MODE == MODE_LIST) {
            // writes stay inside the group's regions sized by the counting walk
            unsigned bs = bl & ~bn;
            long long im = W.off_m + __popc(ba & lt), is = W.off_s + __popc(bs & lt), in = W.off_n + __popc(bn & lt);
            if (acc && im < W.lim_m) P.lm[im] = node;
            if (lf && !nw && is < W.lim_s) P.lr[is] = make_int2(link, cnt);
            if (nw && in < W.lim_n) P.lr[in] = make_int2(link, cnt);
            W.off_m += __popc(ba);
            W.off_s += __popc(bs);
            W.off_n += __popc(bn);
        }
        if (MODE == MODE_LIST1) {
            // staged; what does not fit is counted only
            unsigned bs = bl & ~bn;
            long long im = W.off_m + __popc(ba & lt), is = W.off_s + __popc(bs & lt), in = W.off_n + __popc(bn & lt);
            if (acc && im < W.lim_m) W.sm[im] = node;
            if (lf && !nw && is < W.lim_s) W.ss[is] = make_int2(link, cnt);
            if (nw && in < W.lim_n) W.sn[in] = make_int2(link, cnt);
            W.off_m += __popc(ba);
            W.off_s += __popc(bs);
            W.off_n += __popc(bn);
        }
        return;
    }
    if (MODE == MODE_DUMP) {
        if (acc) P.dbg_m[W.off_m + __popc(ba & lt)] = node;
        if (lf) P.dbg_p[W.off_p + __popc(bl & lt)] = node;
        W.off_m += __popc(ba);
        W.off_p += __popc(bl);
        return;
    }
    if (acc) S.p2m[W.nm + __popc(ba & lt)] = node;
    W.nm += __popc(ba);
    if (lf) S.leafq[(W.qt + __popc(bl & lt)) & 63] = make_int2(link, cnt);
    W.qt += __popc(bl);
    W.qn += lc;
    __syncwarp();
}

// Advance the P2P range queue by cnt particles without staging them.
template <class SM>
__device__ __forceinline__ void skip_p2p(const SM &S, int cnt, int &qh, int &qoff)
{
    int done = 0;
    for (int it = 0; done < cnt && it < 66; it++) {
        int2 hr = S.leafq[qh & 63];
        int take = min(hr.y - qoff, cnt - done);
        if (take < 0) take = 0;
        done += take;
        qoff += take;
        if (qoff >= hr.y) {
            qh++;
            qoff = 0;
        }
    }
}

// Evaluate every full tile (final = false) or everything left (final = true);
// tiles are numbered in walk order and item kk of K evaluates tiles kk mod K.
template <bool QUAD, int MODE>
__device__ __forceinline__ void flush_tiles(const WalkParams &P, WarpSmem &S, WalkState &W, const Tgt &T, int lane,
                                            bool final, int kk, int K)
{
    if (MODE == MODE_COUNT || MODE == MODE_DUMP || MODE == MODE_LIST || MODE == MODE_LIST1) return;
    const int lim = final ? 1 : 32;
    while (MODE == MODE_EVAL64 && W.nm >= lim) {
        int c = min(W.nm, 32);
        if (W.tile++ % K == kk) {
            stage_p2m64<QUAD>(P, S, S.p2m + W.nm - c, c, lane);
            if (T.has) fwd_p2m64<QUAD>(S, c, T, W.dax, W.day, W.daz, W.phi);
            __syncwarp();
        }
        W.nm -= c;
    }
    while (MODE == MODE_EVAL64 && W.qn >= lim) {
        int c = min(W.qn, 32);
        if (W.tile++ % K == kk) {
            stage_p2p64(P, S, c, W.qh, W.qoff, lane);
            if (T.has) fwd_p2p64(S, c, T, W.dax, W.day, W.daz, W.phi);
            __syncwarp();
        } else {
            skip_p2p(S, c, W.qh, W.qoff);
        }
        W.qn -= c;
    }
    while (W.nm >= lim) {
        int c = min(W.nm, 32);
        if (W.tile++ % K == kk) {
            stage_p2m<QUAD, MODE == MODE_VJP>(P, S, S.p2m + W.nm - c, c, T, lane);
            if (MODE == MODE_VJP) vjp_p2m<QUAD>(P, S, c, T, W.c0, W.c1, W.c2, W.cf, W.ax, W.ay, W.az, lane);
            else if (T.has) fwd_p2m<QUAD>(S, c, T, W.ax, W.ay, W.az, W.phi);
            __syncwarp();
        }
        W.nm -= c;
    }
    while (W.qn >= lim) {
        int c = min(W.qn, 32);
        if (W.tile++ % K == kk) {
            stage_p2p(P, S, c, W.qh, W.qoff, T, lane);
            if (MODE == MODE_VJP) vjp_p2p(P, S, c, T, W.c0, W.c1, W.c2, W.cf, W.ax, W.ay, W.az, lane);
            else if (T.has) fwd_p2p(S, c, T, W.ax, W.ay, W.az, W.phi);
            __syncwarp();
        } else {
            skip_p2p(S, c, W.qh, W.qoff);
        }
        W.qn -= c;
    }
}

// One work item: group g, item kk of K.  Every item of a group walks the same
// lists (the walk is cheap next to the evaluation) and evaluates the tiles
// kk, kk + K, ... of the walk order, so the items' work partitions the group's.
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <bool QUAD, int MODE, bool GSTACK>
__device__ void walk_group_body(const WalkParams &P, WarpSmem &S, int2 *stack, int g, int kk, int K, int item,
                                int lane, int wid, int &cloud_out);

// One work item, plus the per-cloud completion time when timing is on.
template <bool QUAD, int MODE, bool GSTACK>
__device__ __forceinline__ void walk_group(const WalkParams &P, WarpSmem &S, int2 *stack, int g, int kk, int K,
                                           int item, int lane, int wid)
{
    int cloud = 0;
    walk_group_body<QUAD, MODE, GSTACK>(P, S, stack, g, kk, K, item, lane, wid, cloud);
    if (P.ctime && lane == 0) atomicMax(&P.ctime[cloud], global_ns());
}

// Targets of group g on the lanes (see Tgt), the group's integer box, its
// largest hq and its cloud.
template <bool F64>
__device__ __forceinline__ void setup_group(const WalkParams &P, int g, int lane, Tgt &T, int glo[3], int ghi[3],
                                            unsigned long long &hq, int &cloud, int &tfirst, int &tcount)
{
    const int2 gt = P.gtab[g];
    tfirst = gt.x;
    tcount = gt.y;
    T.tp = 1;
    while (T.tp < tcount) T.tp <<= 1;
    T.R = 32 / T.tp;
    T.tl = lane & (T.tp - 1);
    T.slice = lane / T.tp;
    T.has = T.tl < tcount;
    T.r = T.has ? P.tgt[tfirst + T.tl] : -1;
    // the group's cloud: its frame, and its root (node id = cloud id)
    cloud = P.pcloud ? P.pcloud[P.tgt[tfirst]] : 0;
    const Frame fr = P.frames[cloud];
    T.s22 = (float)fr.half_cell;
    uint32_t lo[3] = {SFG_GRID_MAX, SFG_GRID_MAX, SFG_GRID_MAX}, hi[3] = {0, 0, 0};
    hq = 0;
    double xd[3] = {0, 0, 0};
    T.h = 1.f;
    T.sink = false;
    if (T.has) {
        uint64_t k = P.key[T.r];
        lo[0] = hi[0] = compact3(k >> 2);
        lo[1] = hi[1] = compact3(k >> 1);
        lo[2] = hi[2] = compact3(k);
        for (int a = 0; a < 3; a++) xd[a] = P.pos_s[3 * (size_t)T.r + a];
        double h = P.soft_s[T.r];
        hq = hq_of(h, fr.scale);
        T.h = (float)h;
        T.sink = P.sink_s[T.r] != 0;
    }
    T.hinv = 1.f / T.h;
    if (F64) {
        for (int a = 0; a < 3; a++) T.x64[a] = xd[a];
        T.h64 = T.has ? P.soft_s[T.r] : 1.0;
        T.hinv64 = 1.0 / T.h64;
    }
    for (int a = 0; a < 3; a++) {
        glo[a] = (int)__reduce_min_sync(FULL, lo[a]);
        ghi[a] = (int)__reduce_max_sync(FULL, hi[a]);
        T.cg[a] = glo[a] + ghi[a] + 1;
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(FULL, hq, o);
        hq = t > hq ? t : hq;
    }
    T.rel = P.gps != nullptr;
    if (T.rel) {
        double gm = T.has ? P.gps[T.r] : __longlong_as_double(0x7ff0000000000000ll);
        for (int o = 16; o > 0; o >>= 1) gm = fmin(gm, __shfl_xor_sync(FULL, gm, o));
        T.rel_ag = __dmul_rn(P.ralpha, gm);
        T.rel_L0 = fr.L0;
        const double cell = ldexp(fr.L0, -SFG_LMAX);
        T.rel_cell2 = __dmul_rn(cell, cell);
        T.rel_agf = (float)T.rel_ag;
        T.rel_GL0f = (float)__dmul_rn(P.rG, __dmul_rn(fr.L0, fr.L0));
        T.rel_cell2f = (float)T.rel_cell2;
    }
    double c0 = fr.x0[0] + (double)T.cg[0] * fr.half_cell;
    double c1 = fr.x0[1] + (double)T.cg[1] * fr.half_cell;
    double c2 = fr.x0[2] + (double)T.cg[2] * fr.half_cell;
    T.ox = (float)(xd[0] - c0);
    T.oy = (float)(xd[1] - c1);
    T.oz = (float)(xd[2] - c2);
}

// Per-target results of one work item (item kk of K of group g): the
// forward field (whole, or a partial sum that the group's last item adds up
// in item order) or the target side of the adjoint; the interaction counts
// once per group.  n_src_p: P2P particles of the group's list (its own
// target included), n_src_m: P2M nodes.
template <int MODE>
__device__ __forceinline__ void finish_targets(const WalkParams &P, const Tgt &T, int g, int kk, int K, int tfirst,
                                               int tcount, float ax, float ay, float az, double phi, int n_src_p,
                                               int n_src_m, int n_src_pn, int lane)
{
    for (int o = T.tp; o < 32; o <<= 1) {
        ax += __shfl_xor_sync(FULL, ax, o);
        ay += __shfl_xor_sync(FULL, ay, o);
        az += __shfl_xor_sync(FULL, az, o);
        phi += __shfl_xor_sync(FULL, phi, o);
    }
    if (MODE == MODE_EVAL || MODE == MODE_TIDAL || MODE == MODE_JERK) {
        if (K == 1) {
            if (T.has && T.slice == 0) {
                P.res_a[tfirst + T.tl] = make_float4(ax, ay, az, 0.f);
                P.res_phi[tfirst + T.tl] = phi;
            }
        } else {
            // partial sums of this item; the group's last item sums them in k order
            const size_t slot = (size_t)(P.soff[g] + kk) * 32;
            if (T.has && T.slice == 0) {
                P.part_a[slot + T.tl] = make_float4(ax, ay, az, 0.f);
                P.part_phi[slot + T.tl] = phi;
            }
            __threadfence();
            __syncwarp();
            int last = 0;
            if (lane == 0) last = atomicAdd(&P.gdone[g], 1) == K - 1;
            last = __shfl_sync(FULL, last, 0);
            if (last) {
                __threadfence();
                if (T.has && T.slice == 0) {
                    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
                    double ph = 0.0;
                    const size_t s0 = (size_t)P.soff[g] * 32;
                    for (int k = 0; k < K; k++) {
                        float4 v = __ldcg(&P.part_a[s0 + (size_t)k * 32 + T.tl]);
                        a.x += v.x;
                        a.y += v.y;
                        a.z += v.z;
                        ph += __ldcg(&P.part_phi[s0 + (size_t)k * 32 + T.tl]);
                    }
                    P.res_a[tfirst + T.tl] = a;
                    P.res_phi[tfirst + T.tl] = ph;
                }
            }
        }
    } else if (MODE == MODE_VJP) {
        if (T.has && T.slice == 0) {
            double *dst = P.gpart + 4 * (size_t)T.r;
            atomicAdd(dst, (double)ax);
            atomicAdd(dst + 1, (double)ay);
            atomicAdd(dst + 2, (double)az);
        }
    }
    if (lane == 0 && kk == 0) {
        // count the group's list once (self pairs excluded)
        atomicAdd(&P.counters[0], (unsigned long long)tcount * (unsigned long long)(n_src_p - 1));
        atomicAdd(&P.counters[1], (unsigned long long)tcount * (unsigned long long)n_src_m);
        if (n_src_pn) atomicAdd(&P.counters[8], (unsigned long long)tcount * (unsigned long long)n_src_pn);
    }
}

// One-pass list walk, end of a group: its list sizes, space reserved in the
// final buffers (every group adds its exact sizes, so the totals size a
// second attempt), and the staged lists copied there if they were staged
// whole and the space is inside the buffers.
__device__ void commit_staged(const WalkParams &P, const WalkState &W, int g, int lane)
{
    const int ns = W.tot_leaf - W.tot_ln, nn = W.tot_ln;
    long long bm = 0, br = 0;
    int ok = 0;
    if (lane == 0) {
        int *c = P.dbg_counts + NCNT * (size_t)g;
        c[0] = W.tot_m;
        c[1] = ns;
        c[2] = W.tot_p - W.tot_pn;
        c[3] = nn;
        c[4] = W.tot_pn;
        bm = (long long)atomicAdd(&P.lbump[0], (unsigned long long)W.tot_m);
        br = (long long)atomicAdd(&P.lbump[1], (unsigned long long)W.tot_leaf);
        atomicAdd(&P.lbump[6], (unsigned long long)W.tot_p);
        atomicMax(&P.lbump[4], (unsigned long long)W.tot_m);
        atomicMax(&P.lbump[5], (unsigned long long)max(ns, nn));
        const bool staged = W.tot_m <= P.stg_cap_m && ns <= P.stg_cap_r && nn <= P.stg_cap_r;
        const bool room = bm + W.tot_m <= P.lcap_m && br + W.tot_leaf <= P.lcap_r;
        ok = staged && room;
        if (room) {
            P.lmo_w[g] = bm;
            P.lro_w[g] = br;
            if (!staged) P.rlist[atomicAdd(&P.lbump[3], 1ull)] = g;
        } else {
            atomicOr(&P.lbump[2], 1ull);
        }
    }
    ok = __shfl_sync(FULL, ok, 0);
    __syncwarp(); // the lanes' staging writes are visible to the copy
    if (ok) {
        bm = __shfl_sync(FULL, bm, 0);
        br = __shfl_sync(FULL, br, 0);
        for (int i = lane; i < W.tot_m; i += 32) P.lm[bm + i] = W.sm[i];
        for (int i = lane; i < ns; i += 32) P.lr[br + i] = W.ss[i];
        for (int i = lane; i < nn; i += 32) P.lr[br + ns + i] = W.sn[i];
    }
    __syncwarp(); // the copy has read the staging before the next group writes it
}

template <bool QUAD, int MODE, bool GSTACK>
__device__ void walk_group_body(const WalkParams &P, WarpSmem &S, int2 *stack, int g, int kk, int K, int item,
                                int lane, int wid, int &cloud_out)
{
    const unsigned lt = (1u << lane) - 1u;
    const int cap = GSTACK ? GSTK : STK;
    Tgt T;
    int glo[3], ghi[3], cloud, tfirst, tcount;
    unsigned long long hq;
    setup_group<MODE == MODE_EVAL64>(P, g, lane, T, glo, ghi, hq, cloud, tfirst, tcount);
    cloud_out = cloud;
    WalkState W;
    W.sp = W.nm = W.qh = W.qt = W.qoff = W.qn = W.tile = 0;
    W.tot_m = W.tot_p = W.tot_leaf = W.tot_ln = W.tot_pn = 0;
    W.off_s = W.off_n = 0;
    W.ax = W.ay = W.az = 0.f;
    W.phi = 0.0;
    W.dax = W.day = W.daz = 0.0;
    W.c0 = W.c1 = W.c2 = W.cf = 0.f;
    W.off_m = W.off_p = 0;
    if (MODE == MODE_VJP && T.has) {
        float4 cv = P.cot[tfirst + T.tl];
        W.c0 = cv.x;
        W.c1 = cv.y;
        W.c2 = cv.z;
        W.cf = cv.w;
    }
    if (MODE == MODE_DUMP) {
        W.off_m = P.dbg_off[2 * g];
        W.off_p = P.dbg_off[2 * g + 1];
    }
    W.lim_m = W.lim_s = W.lim_n = 0;
    if (MODE == MODE_LIST) {
        const int *c = P.lcnt + NCNT * (size_t)g;
        W.off_m = P.lmo[g];
        W.off_s = P.lro[g];
        W.off_n = P.lro[g] + c[1];
        W.lim_m = W.off_m + c[0];
        W.lim_s = W.off_n;
        W.lim_n = W.off_n + c[3];
    }
    if (MODE == MODE_LIST1) {
        W.sm = P.stg_m + (size_t)wid * P.stg_cap_m;
        W.ss = P.stg_r + (size_t)wid * 2 * P.stg_cap_r;
        W.sn = W.ss + P.stg_cap_r;
        W.lim_m = P.stg_cap_m;
        W.lim_s = W.lim_n = P.stg_cap_r;
    }

    if (lane == 0) stack[0] = make_int2(cloud, 1);
    W.sp = 1;
    __syncwarp();

    bool overflow = false;
    // every node is visited at most once per group, so nn + 1 rounds bound the walk
    int rounds = 0;
    const int max_rounds = P.nn + 1;
    while (W.sp > 0) {
        if (++rounds > max_rounds) {
            if (lane == 0) atomicOr(P.status, ST_ETIMEOUT);
            break;
        }
        int node = -1;
        int taken = 0;
        while (taken < 32 && W.sp > 0) {
            int2 top = stack[W.sp - 1];
            int take = min(32 - taken, top.y);
            if (lane >= taken && lane < taken + take) node = top.x + (top.y - take) + (lane - taken);
            taken += take;
            __syncwarp();
            if (take == top.y) W.sp--;
            else if (lane == 0) stack[W.sp - 1].y = top.y - take;
            __syncwarp();
        }
        bool acc, lf, op, nw;
        int link, cnt;
        test_node(P, T, node, glo, ghi, hq, acc, lf, op, nw, link, cnt);
        unsigned bo = __ballot_sync(FULL, op);
        int npush = __popc(bo);
        if (W.sp + npush > cap) {
            overflow = true;
            break;
        }
        if (op) stack[W.sp + __popc(bo & lt)] = make_int2(link, cnt);
        W.sp += npush;
        append_lists<MODE>(P, S, W, node, acc, lf, nw, link, cnt, lt);
        flush_tiles<QUAD, MODE>(P, S, W, T, lane, false, kk, K);
    }
    if (overflow) {
        if (GSTACK) {
            if (lane == 0) atomicOr(P.status, ST_EOVERFLOW);
        } else if (lane == 0) {
            unsigned long long idx = atomicAdd(&P.counters[2], 1ull);
            P.ovf_list[idx] = item;
        }
        __syncwarp();
        return;
    }
    if (MODE == MODE_COUNT) {
        if (lane == 0) {
            int *c = P.dbg_counts + NCNT * (size_t)g;
            c[0] = W.tot_m;
            c[1] = W.tot_leaf - W.tot_ln;
            c[2] = W.tot_p - W.tot_pn;
            c[3] = W.tot_ln;
            c[4] = W.tot_pn;
        }
        return;
    }
    if (MODE == MODE_LIST1) {
        commit_staged(P, W, g, lane);
        return;
    }
    if (MODE == MODE_DUMP || MODE == MODE_LIST) return;
    flush_tiles<QUAD, MODE>(P, S, W, T, lane, true, kk, K);
    if (MODE == MODE_EVAL64) {
        double dax = W.dax, day = W.day, daz = W.daz, dph = W.phi;
        for (int o = T.tp; o < 32; o <<= 1) {
            dax += __shfl_xor_sync(FULL, dax, o);
            day += __shfl_xor_sync(FULL, day, o);
            daz += __shfl_xor_sync(FULL, daz, o);
            dph += __shfl_xor_sync(FULL, dph, o);
        }
        if (T.has && T.slice == 0) {
            double *dst = P.res64 + 4 * (size_t)(tfirst + T.tl);
            atomicAdd(dst, dax);
            atomicAdd(dst + 1, day);
            atomicAdd(dst + 2, daz);
            atomicAdd(dst + 3, dph);
        }
        if (lane == 0 && kk == 0) {
            atomicAdd(&P.counters[0], (unsigned long long)tcount * (unsigned long long)(W.tot_p - 1));
            atomicAdd(&P.counters[1], (unsigned long long)tcount * (unsigned long long)W.tot_m);
        }
        return;
    }
    finish_targets<MODE>(P, T, g, kk, K, tfirst, tcount, W.ax, W.ay, W.az, W.phi, W.tot_p, W.tot_m, 0, lane);
}

// ------------------------------------------------ stored-list evaluation ----
// The forward and the adjoint evaluate groups from the lists of a prior
// walk (MODE_LIST): P2M node ids, softened P2P particle ranges, Newtonian
// P2P ranges (opened leaves that pass clause (ii), so none of their pairs
// is inside either softening support and none is a self pair).  Item kk of
// K takes a contiguous share of each list's tiles.
struct EvalSmem {
    int2 leafq[64]; // ring of P2P ranges being staged
    float4 tP[32];
    float4 tA[32];
    float tB[32];   // P2M: Qyz; P2P: h^2
    int tN[32];
    // the group's targets, for pairs evaluated off their own lane
    float4 gT[32];  // (ox, oy, oz, h)
    float4 gU[32];  // (1/h, sink flag, target rank bits, h^2)
    float4 sAcc[32]; // per-target sums of the softened pairs: forward (a, phi), adjoint (-dL/dx_i, -)
    union {          // arrays of one mode only
        struct {
            float4 gC[32]; // adjoint: the targets' cotangents (cot_a, cot_phi)
            float4 sS[32]; // adjoint: per-source sums of the softened pairs of a tile (dL/dx_j, dL/dm_j)
        } a;
        struct {
            float sTid[32][8]; // tidal / jerk mode: per-target sums of the softened pairs (as res_T / res_J)
            float4 tV[32];     // jerk / timestep mode: source velocities of the tile
            float4 gV[32];     // jerk / timestep mode: the group's target velocities
        } x;
    } m;
    // the next tile's source records in flight (asynchronous copies): P2P
    // (pw, pc), P2M (E0, E1, E2); each lane copies and later converts its own
    float4 raw[3][32];
    unsigned short sq[1024]; // softened pairs of a tile: target | source << 5
};

constexpr int EVAL_WARPS = 4;
constexpr int EVAL_MINB = 6;

// Particle of this lane in the next cnt particles of the range ring (-1 if
// the ring runs dry, which the callers rule out).
template <class SM>
__device__ __forceinline__ int ring_take(const WalkParams &P, const SM &S, int cnt, int &qh, int &qoff, int lane)
{
    int j = -1, filled = 0;
    for (int it = 0; filled < cnt && it < 66; it++) {
        int2 hr = S.leafq[qh & 63];
        int take = min(hr.y - qoff, cnt - filled);
        if (take < 0) take = 0;
        if (lane >= filled && lane < filled + take) j = hr.x + qoff + (lane - filled);
        filled += take;
        qoff += take;
        if (qoff >= hr.y) {
            qh++;
            qoff = 0;
        }
    }
    if (filled < cnt) {
        if (lane == 0) atomicOr(P.status, ST_ETIMEOUT);
        if (lane >= filled) j = -1;
    }
    return j;
}

template <class SM>
__device__ __forceinline__ void fwd_newt_step(const SM &S, int k, const Tgt &T, float &ax, float &ay, float &az,
                                              float &pt)
{
    float4 p = S.tP[k];
    float dx = p.x - T.ox, dy = p.y - T.oy, dz = p.z - T.oz;
    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float rinv = rsqrtf(r2);
    float mr = p.w * rinv;
    float mr3 = mr * (rinv * rinv);
    ax = fmaf(mr3, dx, ax);
    ay = fmaf(mr3, dy, ay);
    az = fmaf(mr3, dz, az);
    pt -= mr;
}

template <class SM>
__device__ __forceinline__ void fwd_p2p_newt(const SM &S, int cnt, const Tgt &T, float &ax, float &ay, float &az,
                                             double &phi)
{
    float pt = 0.f;
#pragma unroll 2
    for (int k = T.slice; k < cnt; k += T.R) fwd_newt_step(S, k, T, ax, ay, az, pt);
    phi += (double)pt;
}

// Adjoint of a Newtonian tile: the systolic source-side sums of vjp_p2p with
// the Newtonian kernel only.
template <class SM>
__device__ __forceinline__ void vjp_p2p_newt(const WalkParams &P, const SM &S, int cnt, const Tgt &T, float c0,
                                             float c1, float c2, float cf, float &gx, float &gy, float &gz, int lane)
{
    const int TP = T.tp, base = T.slice * TP;
    const int nxt = (T.tl + 1) & (TP - 1);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, am = 0.f;
    for (int jj = 0; jj < TP; jj++) {
        const int k = base + ((T.tl + jj) & (TP - 1));
        if (T.has && k < cnt) {
            float4 p = S.tP[k];
            float dx = p.x - T.ox, dy = p.y - T.oy, dz = p.z - T.oz;
            float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            float rinv = rsqrtf(r2);
            float ri2 = rinv * rinv;
            float K = ri2 * rinv;
            float R = -3.f * K * ri2;
            float m = p.w;
            float cd = fmaf(c0, dx, fmaf(c1, dy, c2 * dz));
            float mK = m * K;
            float sv = m * fmaf(R, cd, cf * K);
            float l0 = fmaf(mK, c0, sv * dx);
            float l1 = fmaf(mK, c1, sv * dy);
            float l2 = fmaf(mK, c2, sv * dz);
            a0 += l0;
            a1 += l1;
            a2 += l2;
            am += fmaf(K, cd, -rinv * cf);
            gx -= l0;
            gy -= l1;
            gz -= l2;
        }
        a0 = __shfl_sync(FULL, a0, nxt, TP);
        a1 = __shfl_sync(FULL, a1, nxt, TP);
        a2 = __shfl_sync(FULL, a2, nxt, TP);
        am = __shfl_sync(FULL, am, nxt, TP);
    }
    const int k = base + T.tl;
    if (k < cnt && S.tN[k] >= 0) {
        double *dst = P.gpart + 4 * (size_t)S.tN[k];
        if (a0 != 0.f) atomicAdd(dst, (double)a0);
        if (a1 != 0.f) atomicAdd(dst + 1, (double)a1);
        if (a2 != 0.f) atomicAdd(dst + 2, (double)a2);
        if (am != 0.f) atomicAdd(dst + 3, (double)am);
    }
}



// Forward of a softened-list tile.  Every pair first takes the Newtonian
// kernel; a pair inside max(h_i, h_j) (the self pair included) is left out
// and flagged in the lane's 32-bit mask instead.  The flagged pairs of the
// whole warp are then compacted into a queue and evaluated with the full
// pair rule 32 at a time, their sums collected per target in shared memory.
template <class SM>
__device__ __forceinline__ void fwd_step_defer(const SM &S, int k, const Tgt &T, float ht2, float &ax, float &ay,
                                               float &az, float &pt, unsigned &mask)
{
    float4 p = S.tP[k];
    float hj2 = S.tB[k];
    float dx = p.x - T.ox, dy = p.y - T.oy, dz = p.z - T.oz;
    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    bool sft = r2 < fmaxf(ht2, hj2);
    if (sft) mask |= 1u << k;
    float rinv = rsqrtf(sft ? 1.f : r2);
    float mr = sft ? 0.f : p.w * rinv;
    float mr3 = mr * (rinv * rinv);
    ax = fmaf(mr3, dx, ax);
    ay = fmaf(mr3, dy, ay);
    az = fmaf(mr3, dz, az);
    pt -= mr;
}

// ---------------------------------------------------------- tidal mode ----
// T = -grad grad Phi (Sec. 2.2) summed on the same lists and with the same
// softened kernel as g (Sec. 2.2.1).  A lane keeps T without its isotropic
// part, t (xx yy zz xy xz yz), and that part's coefficient iso separately:
// T = t - iso I.  A pair adds -m [K I + (dK/dr / r) d d^T] (d = x_j - x_i);
// a node adds the derivative of its monopole (+ quadrupole) field.
struct TidAcc {
    float t[6];
    float iso;
};

__device__ __forceinline__ void tid_add_dd(TidAcc &A, float c, float dx, float dy, float dz)
{
    const float cx = c * dx, cy = c * dy;
    A.t[0] = fmaf(cx, dx, A.t[0]);
    A.t[1] = fmaf(cy, dy, A.t[1]);
    A.t[2] = fmaf(c * dz, dz, A.t[2]);
    A.t[3] = fmaf(cx, dy, A.t[3]);
    A.t[4] = fmaf(cx, dz, A.t[4]);
    A.t[5] = fmaf(cy, dz, A.t[5]);
}

// Jerk of one term of the field a = c d (c = m K(r)), d the source minus the
// target position and w the source minus the target velocity:
// j += c w + m (dK/dr / r) (d . w) d, here for the Newtonian kernel
// (dK/dr / r = -3 K / r^2), mK = m K.  In jerk mode t[0..2] of the extra
// accumulator hold j.
__device__ __forceinline__ void jerk_add(TidAcc &A, float mK, float ri2, float dx, float dy, float dz, float wx,
                                         float wy, float wz)
{
    const float c2 = -3.f * mK * ri2 * fmaf(dx, wx, fmaf(dy, wy, dz * wz));
    A.t[0] = fmaf(mK, wx, fmaf(c2, dx, A.t[0]));
    A.t[1] = fmaf(mK, wy, fmaf(c2, dy, A.t[1]));
    A.t[2] = fmaf(mK, wz, fmaf(c2, dz, A.t[2]));
}

// P2M with its tidal term: monopole -M I / r^3 + 3 M d d^T / r^5; quadrupole
// Q / r^5 - 5 (Qd d^T + d Qd^T) / r^7 - 5/2 q I / r^7 + 35/2 q d d^T / r^9.
// Jerk mode: the node's monopole jerk (Sec. 2.2 sums j from the monopole
// contributions of nodes), with its mass-weighted velocity.
template <int MODE, bool QUAD, class SM>
__device__ __forceinline__ void tid_p2m_step(const SM &S, int k, const Tgt &T, float &ax, float &ay, float &az,
                                             float &pt, TidAcc &A)
{
    float4 p = S.tP[k];
    float dx = p.x - T.ox, dy = p.y - T.oy, dz = p.z - T.oz;
    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float rinv = rsqrtf(r2);
    float ri2 = rinv * rinv;
    float Mri3 = p.w * (ri2 * rinv);
    if (QUAD) {
        float4 q = S.tA[k];
        float qyz = S.tB[k];
        float qzz = -(q.x + q.y);
        float Qd0 = fmaf(q.x, dx, fmaf(q.z, dy, q.w * dz));
        float Qd1 = fmaf(q.z, dx, fmaf(q.y, dy, qyz * dz));
        float Qd2 = fmaf(q.w, dx, fmaf(qyz, dy, qzz * dz));
        float ri5 = rinv * ri2 * ri2;
        float t = fmaf(dx, Qd0, fmaf(dy, Qd1, dz * Qd2)) * ri5; // q / r^5
        float c = fmaf(t, 2.5f * ri2, Mri3);
        ax = fmaf(c, dx, fmaf(-ri5, Qd0, ax));
        ay = fmaf(c, dy, fmaf(-ri5, Qd1, ay));
        az = fmaf(c, dz, fmaf(-ri5, Qd2, az));
        pt = fmaf(-p.w, rinv, fmaf(-0.5f, t, pt));
        if (MODE == MODE_JERK) {
            const float4 v = S.m.x.tV[k];
            jerk_add(A, Mri3, ri2, dx, dy, dz, v.x - T.vx, v.y - T.vy, v.z - T.vz);
            return;
        }
        A.iso += c; // M / r^3 + 5/2 q / r^7
        tid_add_dd(A, fmaf(17.5f * t, ri2 * ri2, 3.f * Mri3 * ri2), dx, dy, dz);
        const float b = -5.f * ri5 * ri2;
        const float e0 = b * Qd0, e1 = b * Qd1, e2 = b * Qd2;
        A.t[0] = fmaf(ri5, q.x, fmaf(2.f * e0, dx, A.t[0]));
        A.t[1] = fmaf(ri5, q.y, fmaf(2.f * e1, dy, A.t[1]));
        A.t[2] = fmaf(ri5, qzz, fmaf(2.f * e2, dz, A.t[2]));
        A.t[3] = fmaf(ri5, q.z, fmaf(e0, dy, fmaf(e1, dx, A.t[3])));
        A.t[4] = fmaf(ri5, q.w, fmaf(e0, dz, fmaf(e2, dx, A.t[4])));
        A.t[5] = fmaf(ri5, qyz, fmaf(e1, dz, fmaf(e2, dy, A.t[5])));
    } else {
        ax = fmaf(Mri3, dx, ax);
        ay = fmaf(Mri3, dy, ay);
        az = fmaf(Mri3, dz, az);
        pt = fmaf(-p.w, rinv, pt);
        if (MODE == MODE_JERK) {
            const float4 v = S.m.x.tV[k];
            jerk_add(A, Mri3, ri2, dx, dy, dz, v.x - T.vx, v.y - T.vy, v.z - T.vz);
            return;
        }
        A.iso += Mri3;
        tid_add_dd(A, 3.f * Mri3 * ri2, dx, dy, dz);
    }
}

template <int MODE, bool QUAD, class SM>
__device__ __forceinline__ void tid_p2m(const SM &S, int cnt, const Tgt &T, float &ax, float &ay, float &az,
                                        double &phi, TidAcc &A)
{
    float pt = 0.f;
    for (int k = T.slice; k < cnt; k += T.R) tid_p2m_step<MODE, QUAD>(S, k, T, ax, ay, az, pt, A);
    phi += (double)pt;
}

// Newtonian pair (every pair of a Newtonian range; the pairs outside both
// supports of a softened range, the others flagged in mask).
template <int MODE, bool SOFT, class SM>
__device__ __forceinline__ void tid_p2p_step(const SM &S, int k, const Tgt &T, float ht2, float &ax, float &ay,
                                             float &az, float &pt, unsigned &mask, TidAcc &A)
{
    float4 p = S.tP[k];
    float dx = p.x - T.ox, dy = p.y - T.oy, dz = p.z - T.oz;
    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    bool sft = false;
    if (SOFT) {
        sft = r2 < fmaxf(ht2, S.tB[k]);
        if (sft) mask |= 1u << k;
    }
    float rinv = rsqrtf(sft ? 1.f : r2);
    float ri2 = rinv * rinv;
    float mr = sft ? 0.f : p.w * rinv;
    float mr3 = mr * ri2;
    ax = fmaf(mr3, dx, ax);
    ay = fmaf(mr3, dy, ay);
    az = fmaf(mr3, dz, az);
    pt -= mr;
    if (MODE == MODE_JERK) {
        const float4 v = S.m.x.tV[k];
        jerk_add(A, mr3, ri2, dx, dy, dz, v.x - T.vx, v.y - T.vy, v.z - T.vz);
        return;
    }
    A.iso += mr3;
    tid_add_dd(A, 3.f * mr3 * ri2, dx, dy, dz);
}

// Exclusive warp prefix of n and the warp total.
__device__ __forceinline__ int warp_excl(int n, int lane, int &total)
{
    int v = n;
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += t;
    }
    total = __shfl_sync(FULL, v, 31);
    return v - n;
}

__device__ __forceinline__ void fwd_p2p_defer(EvalSmem &S, int cnt, const Tgt &T, float &ax, float &ay, float &az,
                                              double &phi, int lane)
{
    float pt = 0.f;
    unsigned mask = 0u;
    const float ht2 = T.h * T.h;
    if (T.has) {
        if (T.R == 1 && cnt == 32) {
#pragma unroll 8
            for (int k = 0; k < 32; k++) fwd_step_defer(S, k, T, ht2, ax, ay, az, pt, mask);
        } else {
#pragma unroll 2
            for (int k = T.slice; k < cnt; k += T.R) fwd_step_defer(S, k, T, ht2, ax, ay, az, pt, mask);
        }
    }
    phi += (double)pt;
    int total;
    int at = warp_excl(__popc(mask), lane, total);
    if (total == 0) return;
    while (mask) {
        const int k = __ffs(mask) - 1;
        mask &= mask - 1;
        S.sq[at++] = (unsigned short)(T.tl | (k << 5));
    }
    __syncwarp();
    for (int b = 0; b < total; b += 32) {
        if (b + lane < total) {
            const unsigned e = S.sq[b + lane];
            const int t = e & 31, k = e >> 5;
            const float4 tg = S.gT[t], tu = S.gU[t];
            const float4 p = S.tP[k], hh = S.tA[k];
            if (__float_as_int(hh.z) != __float_as_int(tu.z)) { // not the self pair
                float dx = p.x - tg.x, dy = p.y - tg.y, dz = p.z - tg.z;
                float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                // pair rule (Sec. 2.2.1): gas-gas averages the kernels of both
                // supports, any sink uses one kernel of the larger support
                bool sink = tu.y != 0.f || hh.w != 0.f;
                bool tbig = tg.w >= hh.x;
                float ha = tbig ? tg.w : hh.x, hainv = tbig ? tu.x : hh.y;
                float hb = sink ? ha : (tbig ? hh.x : tg.w), hbinv = sink ? hainv : (tbig ? hh.y : tu.x);
                float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
                float r = r2 * rinv;
                float K1, P1, K2, P2;
                soft_KP(r, rinv, ha, hainv, K1, P1);
                soft_KP(r, rinv, hb, hbinv, K2, P2);
                float mK = p.w * 0.5f * (K1 + K2);
                atomicAdd(&S.sAcc[t].x, mK * dx);
                atomicAdd(&S.sAcc[t].y, mK * dy);
                atomicAdd(&S.sAcc[t].z, mK * dz);
                atomicAdd(&S.sAcc[t].w, p.w * 0.5f * (P1 + P2));
            }
        }
    }
    __syncwarp();
    // potentials: FP32 within the tile, FP64 across tiles (like the lane sums)
    if (T.has && T.slice == 0) {
        phi += (double)S.sAcc[T.tl].w;
        S.sAcc[T.tl].w = 0.f;
    }
    __syncwarp();
}

// Tidal mode, one P2P tile: Newtonian pairs on the lanes; for a softened
// range the pairs inside max(h_i, h_j) are deferred as in fwd_p2p_defer and
// evaluated with K, P and dK/dr / r of the pair rule.
template <int MODE, bool SOFT>
__device__ __forceinline__ void tid_p2p(EvalSmem &S, int cnt, const Tgt &T, float &ax, float &ay, float &az,
                                        double &phi, TidAcc &A, int lane)
{
    float pt = 0.f;
    unsigned mask = 0u;
    const float ht2 = T.h * T.h;
    if (T.has) {
        for (int k = T.slice; k < cnt; k += T.R) tid_p2p_step<MODE, SOFT>(S, k, T, ht2, ax, ay, az, pt, mask, A);
    }
    phi += (double)pt;
    if (!SOFT) return;
    int total;
    int at = warp_excl(__popc(mask), lane, total);
    if (total == 0) return;
    while (mask) {
        const int k = __ffs(mask) - 1;
        mask &= mask - 1;
        S.sq[at++] = (unsigned short)(T.tl | (k << 5));
    }
    __syncwarp();
    for (int b = 0; b < total; b += 32) {
        if (b + lane < total) {
            const unsigned e = S.sq[b + lane];
            const int t = e & 31, k = e >> 5;
            const float4 tg = S.gT[t], tu = S.gU[t];
            const float4 p = S.tP[k], hh = S.tA[k];
            if (__float_as_int(hh.z) != __float_as_int(tu.z)) { // not the self pair
                float dx = p.x - tg.x, dy = p.y - tg.y, dz = p.z - tg.z;
                float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                bool sink = tu.y != 0.f || hh.w != 0.f;
                bool tbig = tg.w >= hh.x;
                float ha = tbig ? tg.w : hh.x, hainv = tbig ? tu.x : hh.y;
                float hb = sink ? ha : (tbig ? hh.x : tg.w), hbinv = sink ? hainv : (tbig ? hh.y : tu.x);
                float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
                float r = r2 * rinv;
                float K1, P1, R1, K2, P2, R2;
                soft_KPR(r, rinv, ha, hainv, K1, P1, R1);
                soft_KPR(r, rinv, hb, hbinv, K2, P2, R2);
                const float m = p.w;
                const float mK = m * 0.5f * (K1 + K2), mR = m * 0.5f * (R1 + R2);
                atomicAdd(&S.sAcc[t].x, mK * dx);
                atomicAdd(&S.sAcc[t].y, mK * dy);
                atomicAdd(&S.sAcc[t].z, mK * dz);
                atomicAdd(&S.sAcc[t].w, m * 0.5f * (P1 + P2));
                if (MODE == MODE_JERK) {
                    // j += m [K w + (dK/dr / r) (d . w) d]
                    const float4 tv = S.m.x.gV[t], sv = S.m.x.tV[k];
                    const float wx = sv.x - tv.x, wy = sv.y - tv.y, wz = sv.z - tv.z;
                    const float c2 = mR * fmaf(dx, wx, fmaf(dy, wy, dz * wz));
                    atomicAdd(&S.m.x.sTid[t][0], fmaf(mK, wx, c2 * dx));
                    atomicAdd(&S.m.x.sTid[t][1], fmaf(mK, wy, c2 * dy));
                    atomicAdd(&S.m.x.sTid[t][2], fmaf(mK, wz, c2 * dz));
                    continue;
                }
                // T += -m [K I + (dK/dr / r) d d^T]
                atomicAdd(&S.m.x.sTid[t][0], -mR * dx * dx);
                atomicAdd(&S.m.x.sTid[t][1], -mR * dy * dy);
                atomicAdd(&S.m.x.sTid[t][2], -mR * dz * dz);
                atomicAdd(&S.m.x.sTid[t][3], -mR * dx * dy);
                atomicAdd(&S.m.x.sTid[t][4], -mR * dx * dz);
                atomicAdd(&S.m.x.sTid[t][5], -mR * dy * dz);
                atomicAdd(&S.m.x.sTid[t][6], mK);
            }
        }
    }
    __syncwarp();
    if (T.has && T.slice == 0) {
        phi += (double)S.sAcc[T.tl].w;
        S.sAcc[T.tl].w = 0.f;
    }
    __syncwarp();
}

// Adjoint of a softened-list tile: the systolic loop of vjp_p2p_newt with
// the Newtonian kernel for every pair; a pair inside max(h_i, h_j) (the self
// pair included) contributes nothing there and is flagged instead.  The
// flagged pairs of the warp are then evaluated 32 at a time with the full
// pair rule and its tidal tensor, their target-side terms summed per target
// and their source-side terms per source in shared memory; each lane adds
// its source's sums to the systolic ones before the FP64 atomics.
__device__ __forceinline__ void vjp_p2p_defer(const WalkParams &P, EvalSmem &S, int cnt, const Tgt &T, float c0,
                                              float c1, float c2, float cf, float &gx, float &gy, float &gz,
                                              int lane)
{
    const int TP = T.tp, base = T.slice * TP;
    const int nxt = (T.tl + 1) & (TP - 1);
    const float ht2 = T.h * T.h;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, am = 0.f;
    unsigned mask = 0u;
    for (int jj = 0; jj < TP; jj++) {
        const int k = base + ((T.tl + jj) & (TP - 1));
        if (T.has && k < cnt) {
            float4 p = S.tP[k];
            float hj2 = S.tB[k];
            float dx = p.x - T.ox, dy = p.y - T.oy, dz = p.z - T.oz;
            float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            bool sft = r2 < fmaxf(ht2, hj2);
            if (sft) mask |= 1u << k;
            float rinv = rsqrtf(sft ? 1.f : r2);
            float ri2 = rinv * rinv;
            float K = ri2 * rinv;
            float R = -3.f * K * ri2;
            float m = sft ? 0.f : p.w;
            float cd = fmaf(c0, dx, fmaf(c1, dy, c2 * dz));
            float mK = m * K;
            float sv = m * fmaf(R, cd, cf * K);
            float l0 = fmaf(mK, c0, sv * dx);
            float l1 = fmaf(mK, c1, sv * dy);
            float l2 = fmaf(mK, c2, sv * dz);
            a0 += l0;
            a1 += l1;
            a2 += l2;
            am += sft ? 0.f : fmaf(K, cd, -rinv * cf);
            gx -= l0;
            gy -= l1;
            gz -= l2;
        }
        a0 = __shfl_sync(FULL, a0, nxt, TP);
        a1 = __shfl_sync(FULL, a1, nxt, TP);
        a2 = __shfl_sync(FULL, a2, nxt, TP);
        am = __shfl_sync(FULL, am, nxt, TP);
    }
    int total;
    int at = warp_excl(__popc(mask), lane, total);
    const int ks = base + T.tl; // the source whose sums this lane holds
    if (total > 0) {
        S.m.a.sS[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        while (mask) {
            const int k = __ffs(mask) - 1;
            mask &= mask - 1;
            S.sq[at++] = (unsigned short)(T.tl | (k << 5));
        }
        __syncwarp();
        for (int b = 0; b < total; b += 32) {
            if (b + lane < total) {
                const unsigned e = S.sq[b + lane];
                const int t = e & 31, k = e >> 5;
                const float4 tg = S.gT[t], tu = S.gU[t], tc = S.m.a.gC[t];
                const float4 p = S.tP[k], hh = S.tA[k];
                if (__float_as_int(hh.z) != __float_as_int(tu.z)) { // not the self pair
                    float dx = p.x - tg.x, dy = p.y - tg.y, dz = p.z - tg.z;
                    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    // pair rule (Sec. 2.2.1), as in the forward
                    bool sink = tu.y != 0.f || hh.w != 0.f;
                    bool tbig = tg.w >= hh.x;
                    float ha = tbig ? tg.w : hh.x, hainv = tbig ? tu.x : hh.y;
                    float hb = sink ? ha : (tbig ? hh.x : tg.w), hbinv = sink ? hainv : (tbig ? hh.y : tu.x);
                    float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
                    float r = r2 * rinv;
                    float K1, P1, R1, K2, P2, R2;
                    soft_KPR(r, rinv, ha, hainv, K1, P1, R1);
                    soft_KPR(r, rinv, hb, hbinv, K2, P2, R2);
                    float K = 0.5f * (K1 + K2), Pp = 0.5f * (P1 + P2), R = 0.5f * (R1 + R2);
                    float m = p.w;
                    float cd = fmaf(tc.x, dx, fmaf(tc.y, dy, tc.z * dz));
                    float mK = m * K;
                    float sv = m * fmaf(R, cd, tc.w * K);
                    float l0 = fmaf(mK, tc.x, sv * dx);
                    float l1 = fmaf(mK, tc.y, sv * dy);
                    float l2 = fmaf(mK, tc.z, sv * dz);
                    atomicAdd(&S.m.a.sS[k].x, l0);
                    atomicAdd(&S.m.a.sS[k].y, l1);
                    atomicAdd(&S.m.a.sS[k].z, l2);
                    atomicAdd(&S.m.a.sS[k].w, fmaf(K, cd, Pp * tc.w));
                    atomicAdd(&S.sAcc[t].x, -l0);
                    atomicAdd(&S.sAcc[t].y, -l1);
                    atomicAdd(&S.sAcc[t].z, -l2);
                }
            }
        }
        __syncwarp();
        if (ks < cnt) { // padded lanes carry source sums too
            const float4 v = S.m.a.sS[ks];
            a0 += v.x;
            a1 += v.y;
            a2 += v.z;
            am += v.w;
        }
    }
    if (ks < cnt && __float_as_int(S.tA[ks].z) >= 0) {
        double *dst = P.gpart + 4 * (size_t)__float_as_int(S.tA[ks].z);
        if (a0 != 0.f) atomicAdd(dst, (double)a0);
        if (a1 != 0.f) atomicAdd(dst + 1, (double)a1);
        if (a2 != 0.f) atomicAdd(dst + 2, (double)a2);
        if (am != 0.f) atomicAdd(dst + 3, (double)am);
    }
}


// Timestep mode (Sec. 2.3, Delta t_2-body with the minima taken over the
// lists): per target, the smallest t_c^2 = (r^2 + eps^2) / |v_s' - v_s|^2 and
// q = (r^2 + eps^2)^{3/2} / (m_s + m_s') over the tile's sources (t_dyn^2 =
// q / G); eps = max(h_s, h_s') / 2.8 for a particle, h_s / 2.8 for a node
// (its mass combined at its centre of mass, with its mass-weighted velocity).
template <bool NODE, class SM>
__device__ __forceinline__ void ts_tile(const SM &S, int cnt, const Tgt &T, float mt, float &tc2, float &q)
{
    const float eps_n = T.h * (1.f / 2.8f);
    for (int k = T.slice; k < cnt; k += T.R) {
        const float4 p = S.tP[k], v = S.m.x.tV[k];
        float e = eps_n;
        if (!NODE) {
            const float4 hh = S.tA[k];
            if (__float_as_int(hh.z) == T.r) continue; // the target itself
            e = fmaxf(T.h, hh.x) * (1.f / 2.8f);
        }
        const float dx = p.x - T.ox, dy = p.y - T.oy, dz = p.z - T.oz;
        const float wx = v.x - T.vx, wy = v.y - T.vy, wz = v.z - T.vz;
        const float s2 = fmaf(e, e, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        const float dv2 = fmaf(wx, wx, fmaf(wy, wy, wz * wz));
        tc2 = fminf(tc2, __fdividef(s2, dv2));
        q = fminf(q, __fdividef(s2 * sqrtf(s2), mt + p.w));
    }
}

// --------------------------------------------- prefetched tile staging ----
// The evaluation kernel copies the next tile's source records into
// S.raw with asynchronous 16-byte copies (cp.async) while it evaluates the
// current tile, then converts them in place of the synchronous staging
// (same layouts as stage_p2p / stage_p2m).  Each lane
// copies, waits for and converts only its own slot.
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Particle j (this lane's source of a tile of cnt, -1 if none) in flight.
__device__ __forceinline__ void fetch_p2p(const WalkParams &P, EvalSmem &S, int j, int cnt, int lane)
{
    if (lane < cnt && j >= 0 && j < P.npart) {
        cp_async16(&S.raw[0][lane], &P.pw[j]);
        cp_async16(&S.raw[1][lane], &P.pc[j]);
    }
    cp_async_commit();
}

// Convert this lane's fetched particle (softened-range layout, or the
// Newtonian-range layout when NEWT).
template <bool NEWT>
__device__ __forceinline__ void convert_p2p(const WalkParams &P, EvalSmem &S, int j, int cnt, const Tgt &T,
                                            int lane)
{
    if (lane >= cnt) return;
    if (j >= 0 && j < P.npart) {
        const float4 a = S.raw[0][lane];
        const float4 bf = S.raw[1][lane];
        const int bx = __float_as_int(bf.x), by = __float_as_int(bf.y), bz = __float_as_int(bf.z);
        const float px = fmaf((float)(bx - T.cg[0]), T.s22, a.x);
        const float py = fmaf((float)(by - T.cg[1]), T.s22, a.y);
        const float pz = fmaf((float)(bz - T.cg[2]), T.s22, a.z);
        S.tP[lane] = make_float4(px, py, pz, a.w);
        if (NEWT) {
            S.tN[lane] = j;
        } else {
            const float h = bf.w; // negative for a sink
            const float ha = fabsf(h);
            S.tA[lane] = make_float4(ha, 1.f / ha, __int_as_float(j), h < 0.f ? 1.f : 0.f);
            S.tB[lane] = ha * ha;
        }
    } else { // the ring ran dry or a corrupt range: massless and far, no gradient
        atomicOr(P.status, ST_ETIMEOUT);
        S.tP[lane] = make_float4(3e18f, 0.f, 0.f, 0.f);
        if (NEWT) {
            S.tN[lane] = -1;
        } else {
            S.tA[lane] = make_float4(1.f, 1.f, __int_as_float(-1), 0.f);
            S.tB[lane] = 0.f;
        }
    }
}

// Node id (this lane's entry of a P2M tile of cnt) in flight.
__device__ __forceinline__ void fetch_p2m(const WalkParams &P, EvalSmem &S, int id, int cnt, int lane)
{
    if (lane < cnt && (unsigned)id < (unsigned)P.nn) {
        cp_async16(&S.raw[0][lane], &P.E0[id]);
        cp_async16(&S.raw[1][lane], &P.E1[id]);
        cp_async16(&S.raw[2][lane], &P.E2[id]);
    }
    cp_async_commit();
}

template <bool QUAD, bool NODEID>
__device__ __forceinline__ void convert_p2m(const WalkParams &P, EvalSmem &S, int id, int cnt, const Tgt &T,
                                            int lane)
{
    if (lane >= cnt) return;
    if ((unsigned)id < (unsigned)P.nn) {
        const float4 e0 = S.raw[0][lane], e2 = S.raw[2][lane];
        const float px = fmaf((float)(__float_as_int(e2.y) - T.cg[0]), T.s22, e0.x);
        const float py = fmaf((float)(__float_as_int(e2.z) - T.cg[1]), T.s22, e0.y);
        const float pz = fmaf((float)(__float_as_int(e2.w) - T.cg[2]), T.s22, e0.z);
        S.tP[lane] = make_float4(px, py, pz, e0.w);
        if (QUAD) {
            S.tA[lane] = S.raw[1][lane];
            S.tB[lane] = e2.x;
        }
    } else { // not a node (a corrupt list): massless and far, no gradient
        atomicOr(P.status, ST_ETIMEOUT);
        id = -1;
        S.tP[lane] = make_float4(3e18f, 0.f, 0.f, 0.f);
        if (QUAD) {
            S.tA[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
            S.tB[lane] = 0.f;
        }
    }
    if (NODEID) S.tN[lane] = id;
}

// Jerk mode: the velocity of this lane's staged source particle j (or node).
__device__ __forceinline__ void stage_vel(const WalkParams &P, EvalSmem &S, int cnt, int j, int lane)
{
    if (lane < cnt) S.m.x.tV[lane] = (j >= 0 && j < P.npart) ? P.pv[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();
}

// This item's share of one P2P list: nr ranges holding np particles.
template <int MODE, bool NEWT>
__device__ __forceinline__ void eval_p2p_list(const WalkParams &P, EvalSmem &S, const Tgt &T, const int2 *rr, int nr,
                                              int np, int kk, int K, float c0, float c1, float c2, float cf,
                                              float &ax, float &ay, float &az, double &phi, TidAcc &A, int lane)
{
    const int nt = (np + 31) >> 5;
    const int t0 = (int)((long long)nt * kk / K), t1 = (int)((long long)nt * (kk + 1) / K);
    if (t0 >= t1) return;
    const int pb = t0 * 32, pe = min(np, t1 * 32);
    // find the range holding particle pb: 32 ranges at a time, warp prefix sums of their sizes
    int r = -1, qoff = 0, before = 0;
    for (int base = 0; base < nr; base += 32) {
        const int idx = base + lane;
        const int c = idx < nr ? rr[idx].y : 0;
        int incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        unsigned hit = __ballot_sync(FULL, idx < nr && before + incl > pb);
        if (hit) {
            const int L = __ffs(hit) - 1;
            r = base + L;
            qoff = pb - (before + __shfl_sync(FULL, incl - c, L));
            break;
        }
        before += __shfl_sync(FULL, incl, 31);
    }
    if (r < 0) { // the stored sizes disagree with the ranges
        if (lane == 0) atomicOr(P.status, ST_ETIMEOUT);
        return;
    }
    int qh = 0, qt = 0, rn = r;
    // keep >= 32 ranges (or all that are left) queued: a tile spans at most
    // 32; the next batch of ranges is read into a register one refill ahead
    int2 nextr = lane < nr - rn ? rr[rn + lane] : make_int2(0, 0);
    auto refill = [&]() {
        if (qt - qh < 32 && rn < nr) {
            const int k = min(32, nr - rn);
            if (lane < k) S.leafq[(qt + lane) & 63] = nextr;
            qt += k;
            rn += k;
            nextr = lane < nr - rn ? rr[rn + lane] : make_int2(0, 0);
            __syncwarp();
        }
    };
    // the first tile's sources in flight
    refill();
    int jn = ring_take(P, S, min(32, pe - pb), qh, qoff, lane);
    fetch_p2p(P, S, jn, min(32, pe - pb), lane);
    for (int b = pb; b < pe; b += 32) {
        const int c = min(32, pe - b);
        const int j = jn;
        cp_async_wait();
        if (NEWT && MODE != MODE_TSTEP) convert_p2p<true>(P, S, j, c, T, lane);
        else convert_p2p<false>(P, S, j, c, T, lane);
        __syncwarp();
        // the next tile's sources in flight while this one is evaluated
        if (b + 32 < pe) {
            refill();
            const int cn = min(32, pe - b - 32);
            jn = ring_take(P, S, cn, qh, qoff, lane);
            fetch_p2p(P, S, jn, cn, lane);
        }
        constexpr bool EXTRA = MODE == MODE_TIDAL || MODE == MODE_JERK;
        if (MODE == MODE_TSTEP) {
            stage_vel(P, S, c, j, lane);
            if (T.has) ts_tile<false>(S, c, T, T.mt, A.t[0], A.t[1]);
        } else if (NEWT) {
            if (MODE == MODE_JERK) stage_vel(P, S, c, j, lane);
            if (MODE == MODE_VJP) vjp_p2p_newt(P, S, c, T, c0, c1, c2, cf, ax, ay, az, lane);
            else if (EXTRA) tid_p2p<MODE, false>(S, c, T, ax, ay, az, phi, A, lane);
            else if (T.has) fwd_p2p_newt(S, c, T, ax, ay, az, phi);
        } else {
            if (MODE == MODE_JERK) stage_vel(P, S, c, j, lane);
            if (MODE == MODE_VJP) vjp_p2p_defer(P, S, c, T, c0, c1, c2, cf, ax, ay, az, lane);
            else if (EXTRA) tid_p2p<MODE, true>(S, c, T, ax, ay, az, phi, A, lane);
            else fwd_p2p_defer(S, c, T, ax, ay, az, phi, lane);
        }
        __syncwarp();
    }
}


template <bool QUAD, int MODE>
__device__ __forceinline__ int eval_item(const WalkParams &P, EvalSmem &S, int g, int kk, int K, int lane)
{
    Tgt T;
    int glo[3], ghi[3], cloud, tfirst, tcount;
    unsigned long long hq;
    setup_group<false>(P, g, lane, T, glo, ghi, hq, cloud, tfirst, tcount);
    float c0 = 0.f, c1 = 0.f, c2 = 0.f, cf = 0.f;
    if (MODE == MODE_VJP && T.has) {
        float4 cv = P.cot[tfirst + T.tl];
        c0 = cv.x;
        c1 = cv.y;
        c2 = cv.z;
        cf = cv.w;
    }
    float ax = 0.f, ay = 0.f, az = 0.f;
    double phi = 0.0;
    if (T.slice == 0) {
        S.gT[T.tl] = make_float4(T.ox, T.oy, T.oz, T.h);
        S.gU[T.tl] = make_float4(T.hinv, T.sink ? 1.f : 0.f, __int_as_float(T.r), T.h * T.h);
        if (MODE == MODE_VJP) S.m.a.gC[T.tl] = make_float4(c0, c1, c2, cf);
    }
    S.sAcc[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
    TidAcc A = {{0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, 0.f};
    constexpr bool EXTRA = MODE == MODE_TIDAL || MODE == MODE_JERK;
    if (EXTRA) {
#pragma unroll
        for (int c = 0; c < 8; c++) S.m.x.sTid[lane][c] = 0.f;
    }
    T.vx = T.vy = T.vz = 0.f;
    T.mt = 0.f;
    if (MODE == MODE_JERK || MODE == MODE_TSTEP) {
        const float4 v = T.has ? P.pv[T.r] : make_float4(0.f, 0.f, 0.f, 0.f);
        T.vx = v.x;
        T.vy = v.y;
        T.vz = v.z;
        if (T.slice == 0) S.m.x.gV[T.tl] = v;
        if (MODE == MODE_TSTEP) {
            T.mt = T.has ? P.pw[T.r].w : 0.f;
            A.t[0] = A.t[1] = __int_as_float(0x7f800000);
        }
    }
    __syncwarp();
    const int *cn = P.lcnt + NCNT * (size_t)g;
    const int nm = cn[0], nls = cn[1], nps = cn[2], nln = cn[3], npn = cn[4];
    {
        const int *lm = P.lm + P.lmo[g];
        const int nt = (nm + 31) >> 5;
        const int t0 = (int)((long long)nt * kk / K), t1 = (int)((long long)nt * (kk + 1) / K);
        // node ids are read one tile ahead of their records' copies, which run
        // one tile ahead of the evaluation
        auto list_id = [&](int tt) { return (tt < t1 && tt * 32 + lane < nm) ? lm[tt * 32 + lane] : -1; };
        int idn = -1, idnn = -1;
        if (t0 < t1) {
            idn = list_id(t0);
            fetch_p2m(P, S, idn, min(32, nm - t0 * 32), lane);
            idnn = list_id(t0 + 1);
        }
        for (int tt = t0; tt < t1; tt++) {
            const int b = tt * 32, c = min(32, nm - b);
            const int id = idn;
            cp_async_wait();
            convert_p2m<QUAD, MODE == MODE_VJP>(P, S, id, c, T, lane);
            __syncwarp();
            if (tt + 1 < t1) { // the next tile's nodes in flight while this one is evaluated
                idn = idnn;
                fetch_p2m(P, S, idn, min(32, nm - b - 32), lane);
                idnn = list_id(tt + 2);
            }
            if (MODE == MODE_JERK || MODE == MODE_TSTEP) {
                if (lane < c)
                    S.m.x.tV[lane] = (unsigned)id < (unsigned)P.nn ? P.nV[id] : make_float4(0.f, 0.f, 0.f, 0.f);
                __syncwarp();
            }
            if (MODE == MODE_TSTEP) {
                if (T.has) ts_tile<true>(S, c, T, T.mt, A.t[0], A.t[1]);
            } else if (MODE == MODE_VJP) vjp_p2m<QUAD>(P, S, c, T, c0, c1, c2, cf, ax, ay, az, lane);
            else if (EXTRA) {
                if (T.has) tid_p2m<MODE, QUAD>(S, c, T, ax, ay, az, phi, A);
            } else if (T.has) fwd_p2m<QUAD>(S, c, T, ax, ay, az, phi);
            __syncwarp();
        }
    }
    const int2 *lr = P.lr + P.lro[g];
    eval_p2p_list<MODE, false>(P, S, T, lr, nls, nps, kk, K, c0, c1, c2, cf, ax, ay, az, phi, A, lane);
    eval_p2p_list<MODE, true>(P, S, T, lr + nls, nln, npn, kk, K, c0, c1, c2, cf, ax, ay, az, phi, A, lane);
    if (T.has && T.slice == 0) { // the deferred softened pairs' target-side sums
        const float4 v = S.sAcc[T.tl];
        ax += v.x;
        ay += v.y;
        az += v.z;
        if (EXTRA) {
#pragma unroll
            for (int c = 0; c < 6; c++) A.t[c] += S.m.x.sTid[T.tl][c];
            A.iso += S.m.x.sTid[T.tl][6];
        }
    }
    __syncwarp();
    if (MODE == MODE_TSTEP) {
        for (int o = T.tp; o < 32; o <<= 1) {
            A.t[0] = fminf(A.t[0], __shfl_xor_sync(FULL, A.t[0], o));
            A.t[1] = fminf(A.t[1], __shfl_xor_sync(FULL, A.t[1], o));
        }
        if (T.has && T.slice == 0) { // non-negative floats order like their bits
            unsigned *dst = P.res_TS + 2 * (size_t)(tfirst + T.tl);
            atomicMin(dst, __float_as_uint(A.t[0]));
            atomicMin(dst + 1, __float_as_uint(A.t[1]));
        }
    }
    if (MODE == MODE_JERK) {
        for (int o = T.tp; o < 32; o <<= 1) {
#pragma unroll
            for (int c = 0; c < 3; c++) A.t[c] += __shfl_xor_sync(FULL, A.t[c], o);
        }
        if (T.has && T.slice == 0) {
            float *dst = P.res_J + 4 * (size_t)(tfirst + T.tl);
#pragma unroll
            for (int c = 0; c < 3; c++) atomicAdd(dst + c, A.t[c]);
        }
    }
    if (MODE == MODE_TIDAL) {
        // slices -> one sum per target; items of a split group add theirs
        for (int o = T.tp; o < 32; o <<= 1) {
#pragma unroll
            for (int c = 0; c < 6; c++) A.t[c] += __shfl_xor_sync(FULL, A.t[c], o);
            A.iso += __shfl_xor_sync(FULL, A.iso, o);
        }
        if (T.has && T.slice == 0) {
            float *dst = P.res_T + 8 * (size_t)(tfirst + T.tl);
#pragma unroll
            for (int c = 0; c < 6; c++) atomicAdd(dst + c, A.t[c]);
            atomicAdd(dst + 6, A.iso);
        }
    }
    finish_targets<MODE>(P, T, g, kk, K, tfirst, tcount, ax, ay, az, phi, nps + npn, nm, npn, lane);
    return cloud;
}

#include "eval_chunks.cuh"

// Persistent warps take work items (longest first) from an atomic counter.
// resident blocks per SM of the evaluation kernel (the tidal mode carries
// seven more accumulators per lane)
constexpr int TIDAL_MINB = 4;
constexpr int eval_minb(int mode)
{
    return mode == MODE_TIDAL || mode == MODE_JERK || mode == MODE_TSTEP ? TIDAL_MINB : EVAL_MINB;
}

template <bool QUAD, int MODE>
__global__ void __launch_bounds__(EVAL_WARPS * 32, eval_minb(MODE)) k_eval(WalkParams P)
{
    __shared__ EvalSmem sm[EVAL_WARPS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    EvalSmem &S = sm[w];
    const int nwork = P.ioff[*P.d_ngroups];
    if (P.ctime && lane == 0) atomicMin(&P.ctime[P.nclouds], global_ns());
    while (true) {
        int w_i = 0;
        if (lane == 0) w_i = (int)atomicAdd(&P.counters[3], 1ull);
        w_i = __shfl_sync(FULL, w_i, 0);
        if (w_i >= nwork) break;
        const int2 it = P.items[w_i];
        const int cloud = eval_item<QUAD, MODE>(P, S, it.x, it.y, P.kcnt[it.x], lane);
        if (P.ctime && lane == 0) atomicMax(&P.ctime[cloud], global_ns());
    }
}

// Exclusive scans over the groups of the stored-list sizes: lmo (P2M
// entries) and lro (P2P ranges), 64-bit; totals in lmo[ng], lro[ng] and tot[2].
constexpr int LS_NB = 512;

__device__ __forceinline__ long long block_sum64(long long v, long long *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    long long t = 0;
    for (int k = 0; k < nw; k++) t += sh[k];
    return t;
}

__global__ void k_lscan_reduce(const int *cnt, const int *d_ng, long long *bsum)
{
    __shared__ long long sh[32];
    const int ng = *d_ng;
    const int chunk = (ng + LS_NB - 1) / LS_NB;
    const int b0 = min(ng, (int)blockIdx.x * chunk), b1 = min(ng, b0 + chunk);
    long long sm = 0, sr = 0, sp = 0;
    for (int g = b0 + threadIdx.x; g < b1; g += blockDim.x) {
        const int *c = cnt + NCNT * (size_t)g;
        sm += c[0];
        sr += c[1] + c[3];
        sp += (long long)c[2] + c[4];
    }
    sm = block_sum64(sm, sh);
    sr = block_sum64(sr, sh);
    sp = block_sum64(sp, sh);
    if (threadIdx.x == 0) {
        bsum[blockIdx.x] = sm;
        bsum[LS_NB + blockIdx.x] = sr;
        bsum[2 * LS_NB + blockIdx.x] = sp;
    }
}

__global__ void k_lscan_top(long long *bsum, const int *d_ng, long long *lmo, long long *lro, long long *tot)
{
    if (threadIdx.x != 0) return;
    long long rm = 0, rr = 0, rp = 0;
    for (int b = 0; b < LS_NB; b++) {
        long long m = bsum[b], r = bsum[LS_NB + b];
        bsum[b] = rm;
        bsum[LS_NB + b] = rr;
        rm += m;
        rr += r;
        rp += bsum[2 * LS_NB + b];
    }
    const int ng = *d_ng;
    lmo[ng] = rm;
    lro[ng] = rr;
    tot[0] = rm;
    tot[1] = rr;
    tot[2] = rp;
}

__global__ void k_lscan_down(const int *cnt, const int *d_ng, const long long *bsum, long long *lmo, long long *lro)
{
    __shared__ long long shm[32], shr[32];
    const int ng = *d_ng;
    const int chunk = (ng + LS_NB - 1) / LS_NB;
    const int b0 = min(ng, (int)blockIdx.x * chunk), b1 = min(ng, b0 + chunk);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    long long cm = bsum[blockIdx.x], cr = bsum[LS_NB + blockIdx.x];
    for (int base = b0; base < b1; base += blockDim.x) {
        const int g = base + threadIdx.x;
        long long vm = 0, vr = 0;
        if (g < b1) {
            const int *c = cnt + NCNT * (size_t)g;
            vm = c[0];
            vr = c[1] + c[3];
        }
        long long im = vm, ir = vr;
        for (int o = 1; o < 32; o <<= 1) {
            long long tm = __shfl_up_sync(FULL, im, o), tr = __shfl_up_sync(FULL, ir, o);
            if (lane >= o) {
                im += tm;
                ir += tr;
            }
        }
        __syncthreads();
        if (lane == 31) {
            shm[w] = im;
            shr[w] = ir;
        }
        __syncthreads();
        long long pm = 0, pr = 0, tm = 0, tr = 0;
        for (int k = 0; k < nw; k++) {
            if (k < w) {
                pm += shm[k];
                pr += shr[k];
            }
            tm += shm[k];
            tr += shr[k];
        }
        if (g < b1) {
            lmo[g] = cm + pm + im - vm;
            lro[g] = cr + pr + ir - vr;
        }
        cm += tm;
        cr += tr;
    }
}

// flag = 1 if a[0..n) != b[0..n)
__global__ void k_cmp_idx(const int64_t *a, const int64_t *b, int64_t n, int *flag)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        if (a[k] != b[k]) *flag = 1;
}

// The list-only walks (no evaluation) are latency-bound: two more resident
// blocks per SM keep more groups in flight.
__host__ __device__ constexpr int walk_minb(int mode)
{
    return mode == MODE_COUNT || mode == MODE_LIST || mode == MODE_LIST1 ? WALK_MINB + 2 : WALK_MINB;
}

template <bool QUAD, int MODE, bool GSTACK>
__global__ void __launch_bounds__(WALK_WARPS * 32, walk_minb(MODE)) k_walk(WalkParams P)
{
    __shared__ WarpSmem sm[WALK_WARPS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    WarpSmem &S = sm[w];
    int2 *stack = GSTACK ? P.gstack + (size_t)(blockIdx.x * WALK_WARPS + w) * GSTK : S.stack;
    constexpr bool ITEMS = MODE == MODE_EVAL || MODE == MODE_VJP || MODE == MODE_EVAL64;
    // a list-writing walk over the listed groups only (those a one-pass walk could not stage)
    const bool RLIST = MODE == MODE_LIST && P.rlist != nullptr;
    const int ngroups = *P.d_ngroups;
    const int nwork = GSTACK ? (int)P.counters[2] : (ITEMS ? P.ioff[ngroups] : (RLIST ? (int)P.lbump[3] : ngroups));
    if (P.ctime && lane == 0 && !GSTACK) atomicMin(&P.ctime[P.nclouds], global_ns());
    while (true) {
        int w_i = 0;
        if (lane == 0) w_i = (int)atomicAdd(&P.counters[GSTACK ? 4 : 3], 1ull);
        w_i = __shfl_sync(FULL, w_i, 0);
        if (w_i >= nwork) break;
        int item = GSTACK ? P.ovf_list[w_i] : w_i;
        int g = RLIST ? P.rlist[item] : item, kk = 0, K = 1;
        if (ITEMS) {
            int2 it = P.items[item];
            g = it.x;
            kk = it.y;
            K = P.kcnt[g];
        }
        walk_group<QUAD, MODE, GSTACK>(P, S, stack, g, kk, K, item, lane,
                                       (GSTACK ? P.stg_main_warps : 0) + blockIdx.x * WALK_WARPS + w);
    }
}

// Work items from the counted list sizes: the sliced iteration count of a
// group (P2M, softened P2P and Newtonian P2P sources, each weighted by its
// relative cost in quarters: wt = (P2M, softened, Newtonian, walk term),
// times the lane steps a source costs: T'/32 for the tile kernel's T' =
// 2^ceil(log2 T) target lanes, 2/R for the chunk kernels' R slices of
// ceil(T/2) lanes) plus a walk term; groups above the split size are cut
// into up to KMAX items, while the partial-sum slot pool lasts.
constexpr int SPLIT_ITERS = 1024;
constexpr int SPLIT_PER_WARP = 8; // items per resident warp's share, at least
constexpr int KMAX = 32;
constexpr int PSLOTS = 65536;

struct ItemCost {
    int4 wt;    // relative costs (P2M, softened P2P, Newtonian P2P, walk term)
    int chunks; // 1: the chunk kernels' lane layout, 0: the tile kernel's
};

__device__ inline long long group_iters(const int *cnt, int tc, int g, ItemCost ic)
{
    const int4 wt = ic.wt;
    const int *c = cnt + NCNT * (size_t)g;
    const long long src = (long long)wt.x * c[0] + (long long)wt.y * c[2] + (long long)wt.z * c[4];
    const long long walk = ((long long)c[0] + c[1] + c[3]) * wt.w / 16 + 32;
    if (ic.chunks) {
        const int R = 32 / max(1, (tc + 1) / 2);
        return src / (2 * R) + walk;
    }
    int tp = 1;
    while (tp < tc) tp <<= 1;
    return src * tp / 128 + walk;
}

// Total estimated cost of all groups (one 64-bit atomic per warp).
// The share [g0, g1) of the groups a tree evaluates when its calls are split
// across `world` processes (rank `rank` of them): contiguous runs of groups
// in Morton order, by group count.
__host__ __device__ inline void group_share(int ng, int rank, int world, int &g0, int &g1)
{
    g0 = (int)((long long)ng * rank / world);
    g1 = (int)((long long)ng * (rank + 1) / world);
}

__global__ void k_item_total(const int *cnt, const int2 *gtab, const int *d_ngroups, ItemCost wt,
                             unsigned long long *total, int2 share)
{
    int g0, g1;
    group_share(*d_ngroups, share.x, share.y, g0, g1);
    unsigned long long acc = 0;
    for (int g = g0 + blockIdx.x * blockDim.x + threadIdx.x; g < g1; g += gridDim.x * blockDim.x)
        acc += (unsigned long long)group_iters(cnt, gtab[g].y, g, wt);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(total, acc);
}

// Split size: at least SPLIT_ITERS, and at least 1/SPLIT_PER_WARP of one
// resident warp's share of the total, so the split groups need at most ~2
// SPLIT_PER_WARP slots per resident warp (the slot pool holds PSLOTS) and
// every item stays small next to a warp's share (longest-first scheduling
// then balances the rest).
__global__ void k_item_counts(const int *cnt, const int2 *gtab, const int *d_ngroups, ItemCost wt,
                              const unsigned long long *total, long long warps, int *kcnt, int *is_split,
                              int2 share)
{
    int ng = *d_ngroups, g0, g1;
    group_share(ng, share.x, share.y, g0, g1);
    long long C = (long long)(*total / (unsigned long long)(SPLIT_PER_WARP * warps));
    if (C < SPLIT_ITERS) C = SPLIT_ITERS;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        if (g < g0 || g >= g1) { // another process's share: no items
            kcnt[g] = 0;
            is_split[g] = 0;
            continue;
        }
        long long iters = group_iters(cnt, gtab[g].y, g, wt);
        long long k = (iters + C - 1) / C;
        int K = (int)(k < 1 ? 1 : (k > KMAX ? KMAX : k));
        kcnt[g] = K;
        is_split[g] = K > 1 ? K : 0;
    }
}

// Longest first: items are bucketed by log2 of their estimated cost and the
// buckets are issued from the most to the least expensive.
__device__ inline int cost_bucket(const int *cnt, const int2 *gtab, const int *kcnt, int g, ItemCost wt)
{
    long long c = group_iters(cnt, gtab[g].y, g, wt) / kcnt[g];
    int b = 63 - __clzll(c > 1 ? c : 1);
    return 31 - min(b, 31);
}

__global__ void k_item_hist(const int *cnt, const int2 *gtab, const int *kcnt, const int *d_ngroups, ItemCost wt,
                            int *hist)
{
    int ng = *d_ngroups;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x)
        if (kcnt[g] > 0) atomicAdd(&hist[cost_bucket(cnt, gtab, kcnt, g, wt)], kcnt[g]);
}

__global__ void k_item_scan(int *hist)
{
    if (threadIdx.x == 0) {
        int run = 0;
        for (int b = 0; b < 32; b++) {
            int c = hist[b];
            hist[b] = run;
            run += c;
        }
    }
}

__global__ void k_item_fill(const int *cnt, const int2 *gtab, const int *kcnt, const int *d_ngroups, ItemCost wt,
                            int *cursor, int2 *items)
{
    int ng = *d_ngroups;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        int K = kcnt[g];
        if (K == 0) continue;
        int base = atomicAdd(&cursor[cost_bucket(cnt, gtab, kcnt, g, wt)], K);
        for (int k = 0; k < K; k++) items[base + k] = make_int2(g, k);
    }
}

// Split groups past the slot pool stay whole.
__global__ void k_item_cap(const int *soff, const int *d_ngroups, int *kcnt)
{
    int ng = *d_ngroups;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x)
        if (kcnt[g] > 1 && soff[g] + kcnt[g] > PSLOTS) kcnt[g] = 1;
}

// ---------------------------------------------------- group formation ----
// The group level of a cloud holding U targets: the largest L with
// G 8^L <= U (0 below 8 G), the depth at which a uniform cloud's nodes hold
// about G targets.  Nodes above it are always opened and their children are
// not packed together, so that no group spans sparse octants of the top
// levels: such groups had boxes covering much of the cloud, and their
// single-warp walks outlasted the rest of the walk launch.
__device__ __forceinline__ int group_level(int U, int G)
{
    int L = 0;
    for (long long v = 8ll * G; v <= U && L < 21; v *= 8) L++;
    return L;
}
__global__ void k_mark(const int64_t *idx, int64_t n_active, int n, const int32_t *rank, int *flag, int *status)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_active;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx ? idx[k] : k;
        if (i < 0 || i >= n) {
            atomicOr(status, ST_EINVAL);
            continue;
        }
        flag[rank[i]] = 1;
    }
}

__global__ void k_compact(const int *flag, const int *pre, int n, int *tgt)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
        if (flag[r]) tgt[pre[r]] = r;
}

__device__ inline void put_group(int *gflag, int *gcnt, int tf, int tc)
{
    gflag[tf] = 1;
    gcnt[tf] = tc;
}

__global__ void k_group_marks(const int32_t *nfirst, const int32_t *ncount, const int32_t *nchild_first,
                              const int32_t *nnchild, const int32_t *nlevel, const int32_t *ncloud, int nn,
                              int nroots, const int *pre, int G, int *gflag, int *gcnt)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x) {
        int f = nfirst[i];
        int tf = pre[f];
        int c = pre[f + ncount[i]] - tf;
        if (c == 0) continue;
        bool leaf = nnchild[i] == 0;
        const bool root = i < nroots;
        // the cloud's root is node ncloud[i]; its target count sets the group level
        const int rt = ncloud[i];
        const int gl = group_level(pre[nfirst[rt] + ncount[rt]] - pre[nfirst[rt]], G);
        // opened (children considered): more than G targets, or above the group level with children
        const bool open = !leaf && (c > G || nlevel[i] < gl);
        if (root && !open && c <= G) put_group(gflag, gcnt, tf, c);
        if (root && c > G && leaf)
            for (int s = 0; s < c; s += G) put_group(gflag, gcnt, tf + s, min(G, c - s));
        if (!open) continue;
        const bool pack = nlevel[i] >= gl; // siblings are packed together only below it
        int run_first = -1, run_count = 0;
        int cf = nchild_first[i], nc = nnchild[i];
        for (int k = 0; k < nc; k++) {
            int ch = cf + k;
            int ctf = pre[nfirst[ch]];
            int cc = pre[nfirst[ch] + ncount[ch]] - ctf;
            if (cc == 0) continue;
            const bool ch_open = nnchild[ch] > 0 && (cc > G || nlevel[ch] < gl);
            if (cc > G || ch_open) {
                if (run_count) put_group(gflag, gcnt, run_first, run_count);
                run_count = 0;
                if (nnchild[ch] == 0)
                    for (int s = 0; s < cc; s += G) put_group(gflag, gcnt, ctf + s, min(G, cc - s));
                continue;
            }
            if (!pack) {
                put_group(gflag, gcnt, ctf, cc);
                continue;
            }
            if (run_count + cc > G) {
                put_group(gflag, gcnt, run_first, run_count);
                run_count = 0;
            }
            if (run_count == 0) run_first = ctf;
            run_count += cc;
        }
        if (run_count) put_group(gflag, gcnt, run_first, run_count);
    }
}

__global__ void k_group_table(const int *gflag, const int *gcnt, const int *goff, const int *d_U, int2 *gtab)
{
    int U = *d_U;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < U; u += gridDim.x * blockDim.x)
        if (gflag[u]) gtab[goff[u]] = make_int2(u, gcnt[u]);
}

__global__ void k_rows_out(const int64_t *idx, int64_t n_active, int n, const int32_t *rank, const int *pre,
                           const float4 *res_a, const double *res_phi, double G, double *accel, double *phi)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_active;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx ? idx[k] : k;
        if (i < 0 || i >= n) continue;
        int u = pre[rank[i]];
        float4 a = res_a[u];
        accel[3 * k] = G * (double)a.x;
        accel[3 * k + 1] = G * (double)a.y;
        accel[3 * k + 2] = G * (double)a.z;
        if (phi) phi[k] = G * res_phi[u];
    }
}

// Tidal rows in the caller's order: T = G (t - iso I), FP64.
__global__ void k_rows_out_tidal(const int64_t *idx, int64_t n_active, int n, const int32_t *rank, const int *pre,
                                 const float *res_T, double G, double *tidal)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_active;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx ? idx[k] : k;
        if (i < 0 || i >= n) continue;
        const float *r = res_T + 8 * (size_t)pre[rank[i]];
        const double iso = (double)r[6];
        for (int c = 0; c < 6; c++) tidal[6 * k + c] = G * ((double)r[c] - (c < 3 ? iso : 0.0));
    }
}

// Tidal timestep sqrt(eta) (|T|_F^2 / 6)^(-1/4) (Sec. 2.3); +inf where T = 0.
__global__ void k_tidal_dt(const double *tidal, int64_t n, double eta, double *dt)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const double *T = tidal + 6 * k;
        double f2 = T[0] * T[0] + T[1] * T[1] + T[2] * T[2] + 2.0 * (T[3] * T[3] + T[4] * T[4] + T[5] * T[5]);
        dt[k] = f2 > 0.0 ? sqrt(eta) * rsqrt(sqrt(f2 / 6.0)) : __longlong_as_double(0x7ff0000000000000ll);
    }
}

__global__ void k_rows_out64(const int64_t *idx, int64_t n_active, int n, const int32_t *rank, const int *pre,
                             const double *res64, double G, double *accel, double *phi)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_active;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx ? idx[k] : k;
        if (i < 0 || i >= n) continue;
        const double *r = res64 + 4 * (size_t)pre[rank[i]];
        accel[3 * k] = G * r[0];
        accel[3 * k + 1] = G * r[1];
        accel[3 * k + 2] = G * r[2];
        if (phi) phi[k] = G * r[3];
    }
}

// --------------------------------------------------------- host side ----
static int grid_for(int64_t n, int bt)
{
    int64_t g = (n + bt - 1) / bt;
    int64_t cap = (int64_t)num_sms() * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

// Per-call workspace carved from one grow-only allocation.
struct Work {
    int *flag, *pre, *tgt, *gflag, *gcnt, *goff, *ovf;
    Scan1P sc;
    int2 *gtab, *gstack;
    float4 *res_a;
    double *res_phi;
    double *res64; // all-FP64 evaluation: [U][4] (a, phi), accumulated
    float *res_T;  // tidal mode: [U][8] = T without its isotropic part (xx yy zz xy xz yz), that part, -; summed
    float *res_J;        // jerk mode: [U][4] = j (x y z), -; summed
    unsigned *res_TS;    // timestep mode: [U][2] = min t_c^2, min (r^2 + eps^2)^{3/2} / (m_s + m_s') (float bits)
    const float4 *pv;    // jerk mode: particle velocities, sorted (FP32)
    const float4 *nV;    // jerk mode: node mass-weighted velocities (FP32 of the FP64 sums)
    // relative opening criterion (off when gps == NULL): |g_prev| per sorted rank, alpha, G
    const double *gps;
    double ralpha, rG;
    int *cnt, *kcnt, *is_split, *soff, *ioff, *gdone, *hist; // cnt: NCNT list sizes per group
    long long *lmo, *lro; // stored lists: first P2M entry / first P2P range of every group (exclusive scans)
    long long *lpo;       // expanded P2P lists: first particle entry of every group
    int2 *items;
    float4 *part_a;
    double *part_phi;
};

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

static int get_work(Tree *t, cudaStream_t s, Work &w)
{
    const size_t n = (size_t)t->n;
    const int retry_warps = num_sms() * WALK_WARPS;
    const size_t NB = 25;
    size_t sz[NB] = {n * 4, (n + 1) * 4, n * 4, n * 4, n * 4, (n + 1) * 4, (n + PSLOTS) * 4, scan1p_bytes((int)n),
                     n * 8, (size_t)retry_warps * GSTK * 8, n * 16, n * 8,
                     n * 4 * NCNT, n * 4, n * 4, (n + 1) * 4, (n + 1) * 4, n * 4,
                     (size_t)PSLOTS * 32 * 16, (size_t)PSLOTS * 32 * 8, 64 * 4, (n + PSLOTS) * 8,
                     (n + 1) * 8, (n + 1) * 8, (n + 1) * 8};
    size_t total = 0;
    for (size_t b : sz) total += align_up(b);
    bool fresh = false;
    if (t->ws_bytes < total) {
        // allocated while a stream is captured, the workspace would belong to
        // the graph: one call of the tree must come before capture
        if (capturing(s)) return SFG_EINVAL;
        fresh = true;
        t->lists_ok = false; // the list sizes lived in the old workspace
        if (t->ws) dev_free(t, t->ws, s);
        t->ws = dev_alloc(t, total, s);
        if (!t->ws) {
            t->ws_bytes = 0;
            return SFG_ENOMEM;
        }
        t->ws_bytes = total;
    }
    char *p = (char *)t->ws;
    void *ptr[NB];
    for (size_t k = 0; k < NB; k++) {
        ptr[k] = p;
        p += align_up(sz[k]);
    }
    w.flag = (int *)ptr[0];
    w.pre = (int *)ptr[1];
    w.tgt = (int *)ptr[2];
    w.gflag = (int *)ptr[3];
    w.gcnt = (int *)ptr[4];
    w.goff = (int *)ptr[5];
    w.ovf = (int *)ptr[6];
    w.sc.attach(ptr[7], (int)n);
    if (fresh) SFG_CUDA_OK(cudaMemsetAsync(ptr[7], 0, scan1p_bytes((int)n), s)); // zero between scans from here on
    w.gtab = (int2 *)ptr[8];
    w.gstack = (int2 *)ptr[9];
    w.res_a = (float4 *)ptr[10];
    w.res_phi = (double *)ptr[11];
    w.cnt = (int *)ptr[12];
    w.kcnt = (int *)ptr[13];
    w.is_split = (int *)ptr[14];
    w.soff = (int *)ptr[15];
    w.ioff = (int *)ptr[16];
    w.gdone = (int *)ptr[17];
    w.part_a = (float4 *)ptr[18];
    w.part_phi = (double *)ptr[19];
    w.hist = (int *)ptr[20];
    w.items = (int2 *)ptr[21];
    w.lmo = (long long *)ptr[22];
    w.lro = (long long *)ptr[23];
    w.lpo = (long long *)ptr[24];
    return SFG_OK;
}

// Groups of the active set: flags by sorted rank, distinct targets in Morton
// order, group table.  Leaves the group count at w.goff[U] (device).
static int form_groups(Tree *t, const int64_t *active, int64_t n_active, Work &w, const int **d_ngroups,
                       cudaStream_t s)
{
    const int n = (int)t->n, BT = 256;
    SFG_CUDA_OK(cudaMemsetAsync(w.flag, 0, sizeof(int) * (size_t)n, s));
    SFG_CUDA_OK(cudaMemsetAsync(w.gflag, 0, sizeof(int) * (size_t)n, s));
    t->n_launch += 6; // mark, scan, compact, marks, scan, table
    k_mark<<<grid_for(n_active, BT), BT, 0, s>>>(active, n_active, n, t->rank, w.flag, t->d_status);
    w.sc.exclusive(w.flag, w.pre, t->d_n, n, t->d_status, s);
    k_compact<<<grid_for(n, BT), BT, 0, s>>>(w.flag, w.pre, n, w.tgt);
    k_group_marks<<<grid_for(t->nn, BT), BT, 0, s>>>(t->nfirst, t->ncount, t->nchild_first, t->nnchild, t->nlevel,
                                                     t->ncloud, t->nn, t->nclouds, w.pre, t->prm.group_size,
                                                     w.gflag, w.gcnt);
    w.sc.exclusive(w.gflag, w.goff, w.pre + n, n, t->d_status, s);
    k_group_table<<<grid_for(n, BT), BT, 0, s>>>(w.gflag, w.gcnt, w.goff, w.pre + n, w.gtab);
    *d_ngroups = nullptr;
    return SFG_OK;
}

// groups = goff[U] -> counters[5] (as int), U -> counters[6]
__global__ void k_ngroups(const int *pre, int n, const int *goff, unsigned long long *counters)
{
    int U = pre[n];
    *(int *)(counters + 5) = goff[U];
    counters[6] = (unsigned long long)U;
}

static void fill_params(Tree *t, Work &w, WalkParams &P)
{
    P.W0 = t->W0;
    P.W1 = t->W1;
    P.W2 = t->W2;
    P.nfirst = t->nfirst;
    P.ncount = t->ncount;
    P.Whq = t->Whq;
    P.E0 = t->E0;
    P.E1 = t->E1;
    P.E2 = t->E2;
    P.pw = t->pw;
    P.pc = t->pc;
    P.key = t->key;
    P.pos_s = t->pos_s;
    P.soft_s = t->soft_s;
    P.mass_s = t->mass_s;
    P.nM = t->nM;
    P.ncom = t->ncom;
    P.nQ = t->nQ;
    P.res64 = nullptr;
    P.sink_s = t->sink_s;
    P.frames = t->d_frame;
    P.pcloud = t->pcloud;
    P.nclouds = t->nclouds;
    P.ctime = nullptr;
    P.nn = t->nn;
    P.npart = (int)t->n;
    const double th = t->prm.theta;
    for (int l = 0; l <= SFG_LMAX; l++) {
        double v = ldexp(1.0, 2 * (SFG_LMAX - l)) / (th * th);
        P.T[l] = (v < 4611686018427387904.0) ? (unsigned long long)ceil(v) : SFG_CAP62;
    }
    P.gps = t->rel_on ? t->gps : nullptr;
    P.ralpha = t->rel_alpha;
    P.rG = t->prm.G;
    P.gtab = w.gtab;
    P.tgt = w.tgt;
    P.res_a = w.res_a;
    P.res_phi = w.res_phi;
    P.counters = t->d_counters;
    P.ovf_list = w.ovf;
    P.status = t->d_status;
    P.gstack = w.gstack;
    P.dbg_counts = nullptr;
    P.dbg_off = nullptr;
    P.dbg_m = nullptr;
    P.dbg_p = nullptr;
    P.cot = nullptr;
    P.gpart = nullptr;
    P.gnode = nullptr;
    P.lcnt = w.cnt;
    P.lmo = w.lmo;
    P.lro = w.lro;
    P.lm = t->lm;
    P.lr = t->lr;
    P.lp = t->lp;
    P.lpo = w.lpo;
    P.stg_m = nullptr;
    P.stg_r = nullptr;
    P.stg_cap_m = P.stg_cap_r = P.stg_main_warps = 0;
    P.lcap_m = P.lcap_r = 0;
    P.lbump = nullptr;
    P.lmo_w = P.lro_w = nullptr;
    P.rlist = nullptr;
}

template <int MODE>
static void launch_walk(Tree *t, WalkParams &P, cudaStream_t s)
{
    t->n_launch += 2;
    const int blocks = num_sms() * walk_minb(MODE);
    const int retry_blocks = num_sms();
    if (t->prm.quadrupole) {
        k_walk<true, MODE, false><<<blocks, WALK_WARPS * 32, 0, s>>>(P);
        k_walk<true, MODE, true><<<retry_blocks, WALK_WARPS * 32, 0, s>>>(P);
    } else {
        k_walk<false, MODE, false><<<blocks, WALK_WARPS * 32, 0, s>>>(P);
        k_walk<false, MODE, true><<<retry_blocks, WALK_WARPS * 32, 0, s>>>(P);
    }
}

// counters: [0] p2p [1] p2m [2] overflow count [3] work [4] retry work [5] ngroups (int)
// reuse_groups: the workspace still holds the groups of this active set (the
// last groups formed, for the kept lists): take them as they are.
static int prepare(Tree *t, const int64_t *active, int64_t n_active, Work &w, WalkParams &P, cudaStream_t s,
                   bool reuse_groups = false)
{
    const size_t ws_before = t->ws_bytes;
    int rc = get_work(t, s, w);
    if (rc) return rc;
    if (t->ws_bytes != ws_before) reuse_groups = false; // a new workspace holds no groups
    SFG_CUDA_OK(cudaMemsetAsync(t->d_counters, 0, NCOUNTERS * sizeof(unsigned long long), s));
    if (!reuse_groups) {
        const int *dng;
        rc = form_groups(t, active, n_active, w, &dng, s);
        if (rc) return rc;
        t->grp_gen++;
    }
    int *d_ngroups = (int *)(t->d_counters + 5);
    k_ngroups<<<1, 1, 0, s>>>(w.pre, (int)t->n, w.goff, t->d_counters);
    t->n_launch += 1;
    fill_params(t, w, P);
    P.d_ngroups = d_ngroups;
    P.ioff = w.ioff;
    P.items = w.items;
    P.kcnt = w.kcnt;
    P.soff = w.soff;
    P.gdone = w.gdone;
    P.part_a = w.part_a;
    P.part_phi = w.part_phi;
    return SFG_OK;
}

__global__ void k_ctime_reset(unsigned long long *ct, int C)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= C; c += gridDim.x * blockDim.x)
        ct[c] = c < C ? 0ull : ~0ull;
}

// Per-cloud completion stamps of the next walk launch (which = 0 forward, 1 adjoint).
static int cloud_timer_begin(Tree *t, int which, cudaStream_t s, WalkParams &P)
{
    const int C = t->nclouds;
    if (!t->d_ctime) {
        if (capturing(s)) return SFG_EINVAL; // see get_work
        t->d_ctime = (unsigned long long *)dev_alloc(t, 2 * sizeof(unsigned long long) * (size_t)(C + 1), s);
        if (!t->d_ctime) return SFG_ENOMEM;
    }
    P.ctime = t->d_ctime + (size_t)which * (C + 1);
    k_ctime_reset<<<(C + 256) / 256, 256, 0, s>>>(P.ctime, C);
    t->n_launch += 1;
    t->ctime_used[which] = true;
    return SFG_OK;
}

// Count the lists of every group (a walk without evaluation), then cut the
// heavy groups into work items.
template <int MODE>
static void launch_walk(Tree *t, WalkParams &P, cudaStream_t s);

// List sizes of every group (a walk without evaluation).
static void count_lists(Tree *t, Work &w, WalkParams &P, cudaStream_t s)
{
    // a group whose walk gives up (status set) keeps empty lists
    cudaMemsetAsync(w.cnt, 0, sizeof(int) * NCNT * (size_t)t->n, s);
    P.dbg_counts = w.cnt;
    launch_walk<MODE_COUNT>(t, P, s);
    P.dbg_counts = nullptr;
}

// Relative costs (in quarters) of a P2M, softened P2P and Newtonian P2P
// source per target lane, and of the walk term: the chunk kernel's adjoint
// (from its instruction counts per pair: P2M 2.75 times a Newtonian pair, a
// softened-range pair 1.25 times with its checks and deferred pairs), the
// stored-list forward and tile modes (measured per interaction on a clumpy
// cloud) and the walking evaluation (unit weights).  The forward keeps the
// tile layout's split: its items also cut the list expansion, which the
// finer chunk-layout split made slower (0.94 -> 1.24 ms on the paper-scale
// cloud) for no gain in the forward evaluation itself.
constexpr int4 WT_VJP = {11, 5, 4, 1};
constexpr int4 WT_EVAL = {7, 8, 4, 1};
constexpr int4 WT_WALK = {4, 4, 4, 4};

// Cut the heavy groups into work items, from the list sizes.
static void items_from_counts(Tree *t, Work &w, WalkParams &P, cudaStream_t s, int4 weights, bool chunks = false)
{
    const ItemCost wt = {weights, chunks ? 1 : 0};
    const int n = (int)t->n, BT = 256;
    const int *d_ng = P.d_ngroups;
    cudaMemsetAsync(t->d_counters + 2, 0, 3 * sizeof(unsigned long long), s);
    unsigned long long *total = t->d_counters + 7;
    cudaMemsetAsync(total, 0, sizeof(unsigned long long), s);
    const int2 share = make_int2(t->share_rank, t->share_world);
    k_item_total<<<grid_for(n, BT), BT, 0, s>>>(w.cnt, w.gtab, d_ng, wt, total, share);
    const long long warps = (long long)num_sms() * WALK_MINB * WALK_WARPS;
    k_item_counts<<<grid_for(n, BT), BT, 0, s>>>(w.cnt, w.gtab, d_ng, wt, total, warps, w.kcnt, w.is_split,
                                                  share);
    w.sc.exclusive(w.is_split, w.soff, d_ng, n, t->d_status, s);
    k_item_cap<<<grid_for(n, BT), BT, 0, s>>>(w.soff, d_ng, w.kcnt);
    w.sc.exclusive(w.kcnt, w.ioff, d_ng, n, t->d_status, s);
    cudaMemsetAsync(w.gdone, 0, sizeof(int) * (size_t)n, s);
    cudaMemsetAsync(w.hist, 0, 32 * sizeof(int), s);
    if (t->share_world > 1) { // rows of other processes' groups come out as zeros
        cudaMemsetAsync(w.res_a, 0, sizeof(float4) * (size_t)n, s);
        cudaMemsetAsync(w.res_phi, 0, sizeof(double) * (size_t)n, s);
    }
    k_item_hist<<<grid_for(n, BT), BT, 0, s>>>(w.cnt, w.gtab, w.kcnt, d_ng, wt, w.hist);
    k_item_scan<<<1, 32, 0, s>>>(w.hist);
    k_item_fill<<<grid_for(n, BT), BT, 0, s>>>(w.cnt, w.gtab, w.kcnt, d_ng, wt, w.hist, w.items);
    t->n_launch += 8; // total, counts, scan, cap, scan, hist, bin scan, fill
}

static void make_items(Tree *t, Work &w, WalkParams &P, cudaStream_t s)
{
    count_lists(t, w, P, s);
    items_from_counts(t, w, P, s, WT_WALK);
}

// Stored lists are used unless disabled, in the all-FP64 mode, or while the
// stream is captured into a CUDA graph (sizing them synchronizes).
static bool use_lists(const Tree *t, cudaStream_t s)
{
    return t->prm.store_lists != 0 && t->prm.precision == 0 && !capturing(s);
}

static int grow_buffer(Tree *t, void **buf, long long *cap, long long need, size_t elem, cudaStream_t s)
{
    if (*buf && need <= *cap) return SFG_OK;
    if (*buf) dev_free(t, *buf, s);
    const long long c = need + need / 4 > 1024 ? need + need / 4 : 1024;
    *buf = dev_alloc(t, elem * (size_t)c, s);
    if (!*buf) {
        *cap = 0;
        return SFG_ENOMEM;
    }
    *cap = c;
    return SFG_OK;
}

// Process-wide sizing hints of the one-pass list walk: list entries per
// active row in the last lists built (the final buffers are sized from them,
// with a margin) and the per-warp staging capacities (the largest lists of
// a group in the last one-pass walk, with a margin, within bounds).
struct ListHint {
    double m_per = 0.0, r_per = 0.0;
    int stg_m = 4096, stg_r = 1024;
};
static std::mutex g_hint_mu;
static ListHint g_hint;
constexpr int LBUMP = 8; // list reservations and totals ([6]: P2P particle entries, [7]: expansion cursor)
constexpr int STG_MIN_M = 1024, STG_MIN_R = 256, STG_MAX_M = 1 << 16, STG_MAX_R = 1 << 14;

static void update_hint(long long tot_m, long long tot_r, int64_t n_active, long long max_m, long long max_r)
{
    std::lock_guard<std::mutex> lk(g_hint_mu);
    const double na = (double)std::max<int64_t>(n_active, 1);
    g_hint.m_per = (double)tot_m / na;
    g_hint.r_per = (double)tot_r / na;
    if (max_m >= 0) {
        g_hint.stg_m = (int)std::min<long long>(std::max<long long>(max_m + max_m / 4 + 32, STG_MIN_M), STG_MAX_M);
        g_hint.stg_r = (int)std::min<long long>(std::max<long long>(max_r + max_r / 4 + 32, STG_MIN_R), STG_MAX_R);
    }
}

// Lists of every group (P2M node ids, softened and Newtonian P2P ranges) in
// the tree's grow-only buffers.  One walk stages each group's lists per warp
// and copies them to space it reserves; one synchronization then reads the
// reservations.  Groups whose lists outgrew the staging have their space
// reserved all the same, and a list-writing walk of just those groups fills
// it (the next call's staging fits this call's largest lists).  If
// the buffers, sized from the hint, were short, the walk's exact sizes
// place every group's lists contiguously and a second walk writes them.
// Without a hint (the first lists of the process) a counting walk gives the
// sizes instead of the one-pass walk.
// Expanded P2P lists: every group's softened, then Newtonian, particle
// ranges written out as sorted particle ranks, so that the evaluation stages
// a source with one index load.  k_lp_offsets reserves each group's space
// (one atomic per group); k_expand_p2p then fills it one work item per warp,
// each item its share of both lists (the split that balances the
// evaluation balances this pass too: a few groups in dense clumps hold lists
// of thousands of ranges).
__global__ void k_lp_offsets(const int *cnt, const int *d_ng, long long *lpo, unsigned long long *bump, long long cap,
                             int *status)
{
    const int ng = *d_ng;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        const int *c = cnt + NCNT * (size_t)g;
        const long long np = (long long)c[2] + c[4];
        const long long off = (long long)atomicAdd(bump, (unsigned long long)np);
        if (off + np > cap) {
            atomicOr(status, ST_ETIMEOUT);
            lpo[g] = -1;
        } else {
            lpo[g] = off;
        }
    }
}

// Write particles [e0, e1) of a range list (nr ranges) to dst[e0..e1).
__device__ __forceinline__ void expand_share(const int2 *rr, int nr, int e0, int e1, int *dst, int lane, int *status)
{
    if (e0 >= e1) return;
    // the range holding particle e0 (warp-wide prefix search, 32 ranges at a time)
    int r = -1, before = 0;
    for (int base = 0; base < nr && r < 0; base += 32) {
        const int idx = base + lane;
        const int c = idx < nr ? rr[idx].y : 0;
        int incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        const unsigned hit = __ballot_sync(FULL, idx < nr && before + incl > e0);
        if (hit) {
            const int L = __ffs(hit) - 1;
            r = base + L;
            before += __shfl_sync(FULL, incl - c, L);
        } else {
            before += __shfl_sync(FULL, incl, 31);
        }
    }
    if (r < 0) { // the stored sizes disagree with the ranges
        if (lane == 0) atomicOr(status, ST_ETIMEOUT);
        return;
    }
    // ranges r, r + 1, ... starting at particle 'before', 32 at a time: each
    // lane writes every 32nd output of the batch's span and finds its range by
    // a binary search over the batch's list positions
    for (int base = r; base < nr && before < e1; base += 32) {
        const int idx = base + lane;
        const int2 q = idx < nr ? rr[idx] : make_int2(0, 0);
        int incl = q.y;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        const int start = before + incl - q.y; // list position of this lane's range
        const int nb = min(32, nr - base);
        const int end = before + __shfl_sync(FULL, incl, 31);
        const int lo = max(before, e0), hi = min(end, e1);
        for (int eb = lo; eb < hi; eb += 32) {
            const int e = eb + lane;
            int k = 0; // the last range of the batch starting at or before e
            for (int step = 16; step >= 1; step >>= 1) {
                const int c = k + step;
                const int sc = __shfl_sync(FULL, start, c & 31);
                if (c < nb && sc <= e) k = c;
            }
            const int first = __shfl_sync(FULL, q.x, k), st = __shfl_sync(FULL, start, k);
            if (e < hi) dst[e] = first + (e - st);
        }
        before = end;
    }
}

__global__ void k_expand_p2p(WalkParams P, const int2 *lr, int *lp)
{
    const int lane = threadIdx.x & 31;
    const int nw = (int)((gridDim.x * (size_t)blockDim.x) >> 5);
    const int nwork = P.ioff[*P.d_ngroups];
    for (int w = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5); w < nwork; w += nw) {
        const int2 it = P.items[w];
        const int g = it.x, kk = it.y, K = P.kcnt[g];
        const long long off = P.lpo[g];
        if (off < 0) continue; // no room (reported by k_lp_offsets)
        const int *c = P.lcnt + NCNT * (size_t)g;
        const int2 *rr = lr + P.lro[g];
        int *dst = lp + off;
        for (int list = 0; list < 2; list++) {
            const int np = c[2 + 2 * list];
            const int nt = (np + 31) >> 5;
            const int t0 = (int)((long long)nt * kk / K), t1 = (int)((long long)nt * (kk + 1) / K);
            if (t0 < t1)
                expand_share(list == 0 ? rr : rr + c[1], c[1 + 2 * list], t0 * 32, min(np, t1 * 32),
                             list == 0 ? dst : dst + c[2], lane, P.status);
        }
    }
}

// Expand the stored P2P ranges (np_total particle entries over all groups)
// with the work items of the call.
static int expand_lists(Tree *t, Work &w, WalkParams &P, cudaStream_t s)
{
    if (t->lp_ready) return SFG_OK;
    int rc = grow_buffer(t, (void **)&t->lp, &t->lp_cap, std::max(t->lp_need, 1ll), sizeof(int), s);
    if (rc) return rc;
    SFG_CUDA_OK(cudaMemsetAsync(t->d_lbump + LBUMP - 1, 0, sizeof(unsigned long long), s));
    k_lp_offsets<<<grid_for(t->n, 256), 256, 0, s>>>(w.cnt, P.d_ngroups, w.lpo, t->d_lbump + LBUMP - 1,
                                                      t->lp_cap, t->d_status);
    P.lp = t->lp;
    P.lpo = w.lpo;
    k_expand_p2p<<<num_sms() * 8, 256, 0, s>>>(P, t->lr, t->lp);
    t->n_launch += 2;
    t->lp_ready = true;
    SFG_CUDA_OK(cudaGetLastError());
    return SFG_OK;
}

static int build_lists(Tree *t, Work &w, WalkParams &P, cudaStream_t s, int64_t n_active)
{
    t->lists_ok = false;
    ListHint h;
    {
        std::lock_guard<std::mutex> lk(g_hint_mu);
        h = g_hint;
    }
    if (!t->d_lscan) {
        t->d_lscan = (long long *)dev_alloc(t, sizeof(long long) * (3 * LS_NB + 3), s);
        if (!t->d_lscan) return SFG_ENOMEM;
    }
    if (!t->d_lbump) {
        t->d_lbump = (unsigned long long *)dev_alloc(t, LBUMP * sizeof(unsigned long long), s);
        if (!t->d_lbump) return SFG_ENOMEM;
    }
    const double na = (double)std::max<int64_t>(n_active, 1);
    bool counted = false;
    const int main_warps = num_sms() * walk_minb(MODE_LIST1) * WALK_WARPS;
    const int warps = main_warps + num_sms() * WALK_WARPS;
    const size_t stg_m_bytes = align_up((size_t)warps * h.stg_m * sizeof(int));
    const size_t stg_r_bytes = align_up((size_t)warps * 2 * h.stg_r * sizeof(int2));
    bool one_pass = h.m_per > 0.0;
    if (one_pass) {
        const size_t stg_bytes = stg_m_bytes + stg_r_bytes + sizeof(int) * (size_t)t->n;
        if (t->lstage_bytes < stg_bytes) {
            if (t->lstage) dev_free(t, t->lstage, s);
            t->lstage = dev_alloc(t, stg_bytes, s);
            t->lstage_bytes = t->lstage ? stg_bytes : 0;
        }
        // where the staging or the buffers sized from the hint do not fit in
        // memory, the sizes-first path below allocates exactly what it needs
        one_pass = t->lstage != nullptr &&
                   grow_buffer(t, (void **)&t->lm, &t->lm_cap, (long long)(h.m_per * na * 1.15) + 4096, sizeof(int),
                               s) == SFG_OK &&
                   grow_buffer(t, (void **)&t->lr, &t->lr_cap, (long long)(h.r_per * na * 1.15) + 1024, sizeof(int2),
                               s) == SFG_OK;
    }
    if (one_pass) {
        P.lm = t->lm;
        P.lr = t->lr;
        P.lcap_m = t->lm_cap;
        P.lcap_r = t->lr_cap;
        P.stg_m = (int *)t->lstage;
        P.stg_r = (int2 *)((char *)t->lstage + stg_m_bytes);
        P.rlist = (int *)((char *)t->lstage + stg_m_bytes + stg_r_bytes);
        P.stg_cap_m = h.stg_m;
        P.stg_cap_r = h.stg_r;
        P.stg_main_warps = main_warps;
        P.lbump = t->d_lbump;
        P.lmo_w = w.lmo;
        P.lro_w = w.lro;
        SFG_CUDA_OK(cudaMemsetAsync(t->d_lbump, 0, LBUMP * sizeof(unsigned long long), s));
        SFG_CUDA_OK(cudaMemsetAsync(w.cnt, 0, sizeof(int) * NCNT * (size_t)t->n, s));
        SFG_CUDA_OK(cudaMemsetAsync(t->d_counters + 2, 0, 3 * sizeof(unsigned long long), s));
        P.dbg_counts = w.cnt;
        launch_walk<MODE_LIST1>(t, P, s);
        P.dbg_counts = nullptr;
        unsigned long long b[LBUMP] = {0};
        SFG_CUDA_OK(cudaMemcpyAsync(b, t->d_lbump, sizeof(b), cudaMemcpyDeviceToHost, s));
        SFG_CUDA_OK(cudaStreamSynchronize(s));
        update_hint((long long)b[0], (long long)b[1], n_active, (long long)b[4], (long long)b[5]);
        if (b[2] == 0) {
            if (b[3] > 0) {
                // the groups that outgrew the staging, into their reserved space
                SFG_CUDA_OK(cudaMemsetAsync(t->d_counters + 2, 0, 3 * sizeof(unsigned long long), s));
                launch_walk<MODE_LIST>(t, P, s);
            }
            P.rlist = nullptr;
            t->list_walks = 1;
            t->lp_need = (long long)b[6];
            t->lp_ready = false;
            SFG_CUDA_OK(cudaGetLastError());
            return SFG_OK;
        }
        P.rlist = nullptr;
        counted = true; // the sizes in w.cnt are exact
    }
    if (!counted) count_lists(t, w, P, s);
    long long *tot_d = t->d_lscan + 3 * LS_NB;
    k_lscan_reduce<<<LS_NB, 256, 0, s>>>(w.cnt, P.d_ngroups, t->d_lscan);
    k_lscan_top<<<1, 32, 0, s>>>(t->d_lscan, P.d_ngroups, w.lmo, w.lro, tot_d);
    k_lscan_down<<<LS_NB, 256, 0, s>>>(w.cnt, P.d_ngroups, t->d_lscan, w.lmo, w.lro);
    t->n_launch += 3;
    long long tot[3] = {0, 0, 0};
    SFG_CUDA_OK(cudaMemcpyAsync(tot, tot_d, sizeof(tot), cudaMemcpyDeviceToHost, s));
    SFG_CUDA_OK(cudaStreamSynchronize(s));
    if (!counted) update_hint(tot[0], tot[1], n_active, -1, -1);
    int rc = grow_buffer(t, (void **)&t->lm, &t->lm_cap, tot[0], sizeof(int), s);
    if (rc) return rc;
    rc = grow_buffer(t, (void **)&t->lr, &t->lr_cap, tot[1], sizeof(int2), s);
    if (rc) return rc;
    P.lm = t->lm;
    P.lr = t->lr;
    SFG_CUDA_OK(cudaMemsetAsync(t->d_counters + 2, 0, 3 * sizeof(unsigned long long), s));
    launch_walk<MODE_LIST>(t, P, s);
    t->list_walks = 2;
    t->lp_need = tot[2];
    t->lp_ready = false;
    SFG_CUDA_OK(cudaGetLastError());
    return SFG_OK;
}

// Record the active set the stored lists belong to (and that the groups now
// in the workspace are theirs).
static int remember_active(Tree *t, const int64_t *active, int64_t n_active, cudaStream_t s)
{
    t->lists_grp_gen = t->grp_gen;
    t->la_all = active == nullptr;
    t->la_n = n_active;
    if (active) {
        if (n_active > t->la_cap) {
            if (t->la) dev_free(t, t->la, s);
            t->la = (int64_t *)dev_alloc(t, sizeof(int64_t) * (size_t)n_active, s);
            t->la_cap = t->la ? n_active : 0;
            if (!t->la) return SFG_ENOMEM;
        }
        SFG_CUDA_OK(cudaMemcpyAsync(t->la, active, sizeof(int64_t) * (size_t)n_active, cudaMemcpyDeviceToDevice, s));
    }
    t->lists_ok = true;
    return SFG_OK;
}

// Do the stored lists belong to this active set?  (one synchronization)
static int lists_match(Tree *t, const int64_t *active, int64_t n_active, cudaStream_t s, bool &match)
{
    match = false;
    if (!t->lists_ok || t->la_n != n_active || t->la_all != (active == nullptr)) return SFG_OK;
    if (!active) {
        match = true;
        return SFG_OK;
    }
    if (!t->d_flag) {
        t->d_flag = (int *)dev_alloc(t, sizeof(int), s);
        if (!t->d_flag) return SFG_ENOMEM;
    }
    SFG_CUDA_OK(cudaMemsetAsync(t->d_flag, 0, sizeof(int), s));
    k_cmp_idx<<<grid_for(n_active, 256), 256, 0, s>>>(active, t->la, n_active, t->d_flag);
    t->n_launch += 1;
    int f = 1;
    SFG_CUDA_OK(cudaMemcpyAsync(&f, t->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    SFG_CUDA_OK(cudaStreamSynchronize(s));
    match = f == 0;
    return SFG_OK;
}

// Resident blocks per SM of a kernel at its launch shape (looked up once per
// kernel and device).
template <class F>
static int resident_blocks(F kernel, int threads)
{
    static std::mutex mu;
    static std::vector<std::pair<std::pair<const void *, int>, int>> seen;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_pair((const void *)kernel, dev);
    {
        std::lock_guard<std::mutex> lk(mu);
        for (const auto &e : seen)
            if (e.first == key) return e.second;
    }
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, 0) != cudaSuccess || b < 1) {
        cudaGetLastError();
        b = 1;
    }
    std::lock_guard<std::mutex> lk(mu);
    seen.push_back(std::make_pair(key, b));
    return b;
}

// One persistent launch of a chunked evaluation kernel (quadrupole or
// monopole variant), its grid filling every SM to the kernel's occupancy.
template <int MODE, class FQ, class FM>
static void launch_chunks(FQ kq, FM km, int warps, Tree *t, WalkParams &P, cudaStream_t s)
{
    const int threads = warps * 32;
    if (t->prm.quadrupole) kq<<<num_sms() * resident_blocks(kq, threads), threads, 0, s>>>(P);
    else km<<<num_sms() * resident_blocks(km, threads), threads, 0, s>>>(P);
}

template <int MODE>
static void launch_eval(Tree *t, WalkParams &P, cudaStream_t s)
{
    if constexpr (MODE == MODE_EVAL || MODE == MODE_VJP) {
        // forward and adjoint: source chunks of the tree's depth, two targets per lane
        // (by default 1, the faster depth of both on the paper-scale cloud)
        const int depth = t->prm.list_depth != 0 ? t->prm.list_depth : 1;
        if (depth == 1) launch_chunks<MODE>(ck1::k_eval_chunks<true, MODE>, ck1::k_eval_chunks<false, MODE>,
                                            ck1::CK_WARPS, t, P, s);
        else if (depth == 4) launch_chunks<MODE>(ck4::k_eval_chunks<true, MODE>, ck4::k_eval_chunks<false, MODE>,
                                                 ck4::CK_WARPS, t, P, s);
        else launch_chunks<MODE>(ck2::k_eval_chunks<true, MODE>, ck2::k_eval_chunks<false, MODE>, ck2::CK_WARPS, t,
                                 P, s);
    } else {
        const int blocks = num_sms() * eval_minb(MODE);
        if (t->prm.quadrupole) k_eval<true, MODE><<<blocks, EVAL_WARPS * 32, 0, s>>>(P);
        else k_eval<false, MODE><<<blocks, EVAL_WARPS * 32, 0, s>>>(P);
    }
    t->n_launch += 1;
}

int accel(Tree *t, const int64_t *active, int64_t n_active, double *acc, double *phi, cudaStream_t s)
{
    if (n_active == 0) return SFG_OK;
    Work w;
    WalkParams P;
    ph_begin(t, PH_FWD, s);
    int rc = prepare(t, active, n_active, w, P, s);
    if (rc) return rc;
    const bool f64 = t->prm.precision == 1;
    double *res64 = nullptr;
    if (f64) {
        res64 = (double *)dev_alloc(t, 32 * (size_t)t->n, s);
        if (!res64) return SFG_ENOMEM;
        SFG_CUDA_OK(cudaMemsetAsync(res64, 0, 32 * (size_t)t->n, s));
        P.res64 = res64;
    }
    const bool lists = !f64 && use_lists(t, s);
    if (lists) {
        rc = build_lists(t, w, P, s, n_active);
        if (rc) return rc;
        rc = remember_active(t, active, n_active, s);
        if (rc) return rc;
        items_from_counts(t, w, P, s, WT_EVAL);
        rc = expand_lists(t, w, P, s);
        if (rc) return rc;
    } else {
        t->lists_ok = false; // the counting walk below overwrites their sizes
        make_items(t, w, P, s);
    }
    if (t->timing) {
        int rc2 = cloud_timer_begin(t, 0, s, P);
        if (rc2) return rc2;
    }
    ph_begin(t, PH_FWD_WALK, s);
    if (f64) launch_walk<MODE_EVAL64>(t, P, s);
    else if (lists) launch_eval<MODE_EVAL>(t, P, s);
    else launch_walk<MODE_EVAL>(t, P, s);
    ph_end(t, PH_FWD_WALK, s);
    if (f64) {
        k_rows_out64<<<grid_for(n_active, 256), 256, 0, s>>>(active, n_active, (int)t->n, t->rank, w.pre, res64,
                                                             t->prm.G, acc, phi);
        dev_free(t, res64, s);
    } else {
        k_rows_out<<<grid_for(n_active, 256), 256, 0, s>>>(active, n_active, (int)t->n, t->rank, w.pre, w.res_a,
                                                           w.res_phi, t->prm.G, acc, phi);
    }
    t->n_launch += 1;
    ph_end(t, PH_FWD, s);
    SFG_CUDA_OK(cudaGetLastError());
    return SFG_OK;
}

__global__ void k_gather_sorted(const double *g, const int32_t *order, int n, double *gs)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) gs[r] = g[order[r]];
}

int set_relative(Tree *t, const double *g_prev, double alpha, cudaStream_t s)
{
    t->lists_ok = false; // lists depend on the opening criterion
    if (!g_prev) {
        t->rel_on = false;
        return SFG_OK;
    }
    if (!t->gps) {
        t->gps = (double *)dev_alloc(t, sizeof(double) * (size_t)t->n, s);
        if (!t->gps) return SFG_ENOMEM;
    }
    k_gather_sorted<<<grid_for(t->n, 256), 256, 0, s>>>(g_prev, t->order, (int)t->n, t->gps);
    t->n_launch += 1;
    t->rel_on = true;
    t->rel_alpha = alpha;
    SFG_CUDA_OK(cudaGetLastError());
    return SFG_OK;
}

// Field, potential and tidal tensor from stored lists (walked here unless the
// lists of the same active set are kept).
int accel_tidal(Tree *t, const int64_t *active, int64_t n_active, double *acc, double *phi, double *tidal,
                cudaStream_t s)
{
    if (n_active == 0) return SFG_OK;
    if (t->prm.precision != 0 || capturing(s)) return SFG_EINVAL;
    Work w;
    WalkParams P;
    ph_begin(t, PH_FWD, s);
    int rc = prepare(t, active, n_active, w, P, s);
    if (rc) return rc;
    bool match = false;
    rc = lists_match(t, active, n_active, s, match);
    if (rc) return rc;
    if (!match) {
        rc = build_lists(t, w, P, s, n_active);
        if (rc) return rc;
        rc = remember_active(t, active, n_active, s);
        if (rc) return rc;
    }
    items_from_counts(t, w, P, s, WT_EVAL);
    const size_t need = 32 * (size_t)t->n;
    if (t->ws3_bytes < need) {
        if (t->ws3) dev_free(t, t->ws3, s);
        t->ws3 = dev_alloc(t, need, s);
        if (!t->ws3) {
            t->ws3_bytes = 0;
            return SFG_ENOMEM;
        }
        t->ws3_bytes = need;
    }
    P.res_T = (float *)t->ws3;
    SFG_CUDA_OK(cudaMemsetAsync(P.res_T, 0, need, s));
    if (t->timing) {
        int rc2 = cloud_timer_begin(t, 0, s, P);
        if (rc2) return rc2;
    }
    ph_begin(t, PH_FWD_WALK, s);
    launch_eval<MODE_TIDAL>(t, P, s);
    ph_end(t, PH_FWD_WALK, s);
    k_rows_out<<<grid_for(n_active, 256), 256, 0, s>>>(active, n_active, (int)t->n, t->rank, w.pre, w.res_a,
                                                       w.res_phi, t->prm.G, acc, phi);
    k_rows_out_tidal<<<grid_for(n_active, 256), 256, 0, s>>>(active, n_active, (int)t->n, t->rank, w.pre, P.res_T,
                                                             t->prm.G, tidal);
    t->n_launch += 2;
    ph_end(t, PH_FWD, s);
    SFG_CUDA_OK(cudaGetLastError());
    return SFG_OK;
}

__global__ void k_fill_u32(unsigned *p, int64_t n, unsigned v)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// ---- jerk mode: velocities of particles (sorted, FP32) and nodes ----
__global__ void k_vel_sorted(const double *vel, const int32_t *order, int n, float4 *pv)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const double *v = vel + 3 * (size_t)order[r];
        pv[r] = make_float4((float)v[0], (float)v[1], (float)v[2], 0.f);
    }
}

// Node momenta in FP64, like the centre of mass: a leaf sums m v over its
// members in sorted order, an internal node its children's in octant order.
__global__ void k_mom_leaf(const double *vel, const int32_t *order, const double *mass_s, const int32_t *nfirst,
                           const int32_t *ncount, const int32_t *nnchild, int nn, double *np)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x) {
        if (nnchild[i] != 0) continue;
        double p[3] = {0.0, 0.0, 0.0};
        for (int k = nfirst[i]; k < nfirst[i] + ncount[i]; k++) {
            const double m = mass_s[k];
            const double *v = vel + 3 * (size_t)order[k];
            for (int a = 0; a < 3; a++) p[a] = p[a] + m * v[a];
        }
        for (int a = 0; a < 3; a++) np[3 * (size_t)i + a] = p[a];
    }
}

__global__ void k_mom_internal(const int32_t *nchild_first, const int32_t *nnchild, int b, int e, double *np)
{
    for (int i = b + blockIdx.x * blockDim.x + threadIdx.x; i < e; i += gridDim.x * blockDim.x) {
        if (nnchild[i] == 0) continue;
        double p[3] = {0.0, 0.0, 0.0};
        for (int q = 0; q < nnchild[i]; q++)
            for (int a = 0; a < 3; a++) p[a] = p[a] + np[3 * (size_t)(nchild_first[i] + q) + a];
        for (int a = 0; a < 3; a++) np[3 * (size_t)i + a] = p[a];
    }
}

__global__ void k_node_vel(const double *np, const double *nM, int nn, float4 *nV)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x) {
        const double M = nM[i];
        const double *p = np + 3 * (size_t)i;
        nV[i] = M > 0.0 ? make_float4((float)(p[0] / M), (float)(p[1] / M), (float)(p[2] / M), 0.f)
                        : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Jerk rows in the caller's order, G applied, FP64.
__global__ void k_rows_out_jerk(const int64_t *idx, int64_t n_active, int n, const int32_t *rank, const int *pre,
                                const float *res_J, double G, double *jerk)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_active;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx ? idx[k] : k;
        if (i < 0 || i >= n) continue;
        const float *r = res_J + 4 * (size_t)pre[rank[i]];
        for (int c = 0; c < 3; c++) jerk[3 * k + c] = G * (double)r[c];
    }
}

// Stored lists for the active set (walked here unless kept), work items, and
// the velocities of particles (sorted, FP32) and nodes (FP64 momentum sums).
// Returns the per-target result slots (16 B each) of the jerk / timestep mode.
static int prepare_vel(Tree *t, const double *vel, const int64_t *active, int64_t n_active, Work &w, WalkParams &P,
                       cudaStream_t s, float **res)
{
    const int n = (int)t->n, nn = t->nn, BT = 256;
    int rc = prepare(t, active, n_active, w, P, s);
    if (rc) return rc;
    bool match = false;
    rc = lists_match(t, active, n_active, s, match);
    if (rc) return rc;
    if (!match) {
        rc = build_lists(t, w, P, s, n_active);
        if (rc) return rc;
        rc = remember_active(t, active, n_active, s);
        if (rc) return rc;
    }
    items_from_counts(t, w, P, s, WT_EVAL);
    // workspace: results [n][4] f32, pv [n] float4, node momenta [nn][3] f64, nV [nn] float4
    const size_t need = align_up(16 * (size_t)n) + align_up(16 * (size_t)n) + align_up(24 * (size_t)nn) +
                        align_up(16 * (size_t)nn);
    if (t->ws4_bytes < need) {
        if (t->ws4) dev_free(t, t->ws4, s);
        t->ws4 = dev_alloc(t, need, s);
        if (!t->ws4) {
            t->ws4_bytes = 0;
            return SFG_ENOMEM;
        }
        t->ws4_bytes = need;
    }
    char *p = (char *)t->ws4;
    *res = (float *)p;
    p += align_up(16 * (size_t)n);
    float4 *pv = (float4 *)p;
    p += align_up(16 * (size_t)n);
    double *np = (double *)p;
    p += align_up(24 * (size_t)nn);
    float4 *nV = (float4 *)p;
    k_vel_sorted<<<grid_for(n, BT), BT, 0, s>>>(vel, t->order, n, pv);
    k_mom_leaf<<<grid_for(nn, 128), 128, 0, s>>>(vel, t->order, t->mass_s, t->nfirst, t->ncount, t->nnchild, nn,
                                                 np);
    t->n_launch += 2;
    for (int l = t->depth - 1; l >= 0; l--) {
        const int b = t->lvl_off[l], e = t->lvl_off[l + 1];
        k_mom_internal<<<grid_for(e - b, 128), 128, 0, s>>>(t->nchild_first, t->nnchild, b, e, np);
        t->n_launch += 1;
    }
    k_node_vel<<<grid_for(nn, BT), BT, 0, s>>>(np, t->nM, nn, nV);
    t->n_launch += 1;
    P.pv = pv;
    P.nV = nV;
    SFG_CUDA_OK(cudaGetLastError());
    return SFG_OK;
}

// Field, potential and jerk (stored lists, like accel_tidal).
int accel_jerk(Tree *t, const double *vel, const int64_t *active, int64_t n_active, double *acc, double *phi,
               double *jerk, cudaStream_t s)
{
    if (n_active == 0) return SFG_OK;
    if (t->prm.precision != 0 || capturing(s)) return SFG_EINVAL;
    const int n = (int)t->n;
    Work w;
    WalkParams P;
    ph_begin(t, PH_FWD, s);
    float *res_J = nullptr;
    int rc = prepare_vel(t, vel, active, n_active, w, P, s, &res_J);
    if (rc) return rc;
    SFG_CUDA_OK(cudaMemsetAsync(res_J, 0, 16 * (size_t)n, s));
    P.res_J = res_J;
    if (t->timing) {
        int rc2 = cloud_timer_begin(t, 0, s, P);
        if (rc2) return rc2;
    }
    ph_begin(t, PH_FWD_WALK, s);
    launch_eval<MODE_JERK>(t, P, s);
    ph_end(t, PH_FWD_WALK, s);
    k_rows_out<<<grid_for(n_active, 256), 256, 0, s>>>(active, n_active, n, t->rank, w.pre, w.res_a, w.res_phi,
                                                       t->prm.G, acc, phi);
    k_rows_out_jerk<<<grid_for(n_active, 256), 256, 0, s>>>(active, n_active, n, t->rank, w.pre, res_J, t->prm.G,
                                                            jerk);
    t->n_launch += 2;
    ph_end(t, PH_FWD, s);
    SFG_CUDA_OK(cudaGetLastError());
    return SFG_OK;
}

// dt = sqrt(eta) / (1 / t_c + 1 / t_dyn) from the per-target minima; a
// minimum left at the +inf sentinel imposes no limit.
__global__ void k_rows_out_tstep(const int64_t *idx, int64_t n_active, int n, const int32_t *rank, const int *pre,
                                 const unsigned *res_TS, double G, double eta, double *dt)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_active;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx ? idx[k] : k;
        if (i < 0 || i >= n) continue;
        const unsigned *r = res_TS + 2 * (size_t)pre[rank[i]];
        const double tc2 = (double)__uint_as_float(r[0]), q = (double)__uint_as_float(r[1]);
        const double inv_tc = isinf(tc2) ? 0.0 : rsqrt(tc2);
        const double inv_td = isinf(q) ? 0.0 : sqrt(G / q);
        dt[k] = sqrt(eta) / (inv_tc + inv_td);
    }
}

int sink_timestep(Tree *t, const double *vel, const int64_t *active, int64_t n_active, double eta, double *dt,
                  cudaStream_t s)
{
    if (n_active == 0) return SFG_OK;
    if (t->prm.precision != 0 || capturing(s)) return SFG_EINVAL;
    const int n = (int)t->n;
    Work w;
    WalkParams P;
    ph_begin(t, PH_FWD, s);
    float *res = nullptr;
    int rc = prepare_vel(t, vel, active, n_active, w, P, s, &res);
    if (rc) return rc;
    P.res_TS = (unsigned *)res;
    k_fill_u32<<<grid_for(2 * (int64_t)n, 256), 256, 0, s>>>(P.res_TS, 2 * (int64_t)n, 0x7f800000u); // +inf
    ph_begin(t, PH_FWD_WALK, s);
    launch_eval<MODE_TSTEP>(t, P, s);
    ph_end(t, PH_FWD_WALK, s);
    k_rows_out_tstep<<<grid_for(n_active, 256), 256, 0, s>>>(active, n_active, n, t->rank, w.pre, P.res_TS,
                                                             t->prm.G, eta, dt);
    t->n_launch += 2;
    ph_end(t, PH_FWD, s);
    SFG_CUDA_OK(cudaGetLastError());
    return SFG_OK;
}

int tidal_timestep(const double *tidal, int64_t n, double eta, double *dt, cudaStream_t s)
{
    if (n <= 0) return SFG_OK;
    k_tidal_dt<<<grid_for(n, 256), 256, 0, s>>>(tidal, n, eta, dt);
    SFG_CUDA_OK(cudaGetLastError());
    return SFG_OK;
}

// ---------------------------------------------------------- adjoint ----
// Cotangent rows summed per distinct target (duplicate rows add).
__global__ void k_cot_rows(const int64_t *idx, int64_t n_active, int n, const int32_t *rank, const int *pre,
                           const double *cot_a, const double *cot_phi, double *cotd)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_active;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx ? idx[k] : k;
        if (i < 0 || i >= n) continue;
        int u = pre[rank[i]];
        atomicAdd(&cotd[4 * (size_t)u], cot_a[3 * k]);
        atomicAdd(&cotd[4 * (size_t)u + 1], cot_a[3 * k + 1]);
        atomicAdd(&cotd[4 * (size_t)u + 2], cot_a[3 * k + 2]);
        if (cot_phi) atomicAdd(&cotd[4 * (size_t)u + 3], cot_phi[k]);
    }
}

__global__ void k_cot_pack(const double *cotd, const int *d_U, float4 *cot)
{
    int U = *d_U;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < U; u += gridDim.x * blockDim.x)
        cot[u] = make_float4((float)cotd[4 * (size_t)u], (float)cotd[4 * (size_t)u + 1],
                             (float)cotd[4 * (size_t)u + 2], (float)cotd[4 * (size_t)u + 3]);
}

// Node gradients (gM, g_com, g_Q sym) -> per-unit-mass form (gM, v = g_com / M,
// g_Q).  A massless node's own centre-of-mass and quadrupole terms vanish
// (its moments do not move to first order when a member's mass leaves zero).
__global__ void k_gnode_unit(double *gnode, const float *gnode32, const double *nM, int nn)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x) {
        double *g = gnode + 10 * (size_t)i;
        const float *g32 = gnode32 + 12 * (size_t)i;
        for (int a = 0; a < 10; a++) g[a] += (double)g32[a];
        double M = nM[i];
        if (M > 0.0) {
            for (int a = 1; a < 4; a++) g[a] /= M;
        } else {
            for (int a = 1; a < 10; a++) g[a] = 0.0;
        }
    }
}

// Top-down, one level at a time: a node's terms, written as a quadratic in a
// member position x about the node's centre of mass,
//   dL/dm_k  += gM + v.(x - c) + 3 (x-c)^T S (x-c) - |x-c|^2 tr S
//   dL/dx_k  += m_k (v + 6 S (x-c) - 2 tr S (x-c)),
// are re-expanded about each child's centre c' = c + d (exact identity).
__device__ __forceinline__ void push_node(double *gnode, const double *ncom, const int32_t *nparent, int c)
{
    int p = nparent[c];
    const double *gp = gnode + 10 * (size_t)p;
    double *gc = gnode + 10 * (size_t)c;
    double d[3];
    for (int a = 0; a < 3; a++) d[a] = ncom[3 * (size_t)c + a] - ncom[3 * (size_t)p + a];
    const double *S = gp + 4; // xx yy zz xy xz yz
    double tr = S[0] + S[1] + S[2];
    double Sd[3] = {S[0] * d[0] + S[3] * d[1] + S[4] * d[2], S[3] * d[0] + S[1] * d[1] + S[5] * d[2],
                    S[4] * d[0] + S[5] * d[1] + S[2] * d[2]};
    double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double dSd = d[0] * Sd[0] + d[1] * Sd[1] + d[2] * Sd[2];
    gc[0] += gp[0] + gp[1] * d[0] + gp[2] * d[1] + gp[3] * d[2] + 3.0 * dSd - dd * tr;
    for (int a = 0; a < 3; a++) gc[1 + a] += gp[1 + a] + 6.0 * Sd[a] - 2.0 * tr * d[a];
    for (int q = 0; q < 6; q++) gc[4 + q] += S[q];
}

__global__ void k_gnode_push(double *gnode, const double *ncom, const int32_t *nparent, int b, int e)
{
    for (int c = b + blockIdx.x * blockDim.x + threadIdx.x; c < e; c += gridDim.x * blockDim.x)
        push_node(gnode, ncom, nparent, c);
}

// Leaves to their members, then unpermute into the caller's order with G.
// The small top levels (1..top) in one block, top-down, a barrier between
// levels (a parent's terms are final before its children take them).
struct PushLevels {
    int off[SFG_LMAX + 3];
};

__global__ void __launch_bounds__(256)
    k_gnode_push_top(double *gnode, const double *ncom, const int32_t *nparent, PushLevels L, int top)
{
    for (int l = 1; l <= top; l++) {
        for (int c = L.off[l] + threadIdx.x; c < L.off[l + 1]; c += blockDim.x) push_node(gnode, ncom, nparent, c);
        __syncthreads();
    }
}

// Leaves to their members.  A member's terms are a polynomial in its offset
// s = x - c from the leaf's centre of mass, evaluated in FP32 (s from the
// stored FP32 offsets of member and centre of mass against the leaf centre)
// and added to the FP64 particle gradients; the node gradients stay FP64
// and gM enters in FP64.
// The leaves' node gradients in FP32 for the members' pass: (v, tr S), S[0..3],
// (S[4], S[5], g_M as two words): 48 B per leaf.
__global__ void k_gleaf_prep(const double *gnode, const int32_t *nnchild, int nn, float4 *gl)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x) {
        if (nnchild[i] != 0) continue;
        const double *g = gnode + 10 * (size_t)i;
        const float S0 = (float)g[4], S1 = (float)g[5], S2 = (float)g[6];
        const long long gm = __double_as_longlong(g[0]);
        gl[3 * (size_t)i] = make_float4((float)g[1], (float)g[2], (float)g[3], S0 + S1 + S2);
        gl[3 * (size_t)i + 1] = make_float4(S0, S1, S2, (float)g[7]);
        gl[3 * (size_t)i + 2] =
            make_float4((float)g[8], (float)g[9], __int_as_float((int)gm), __int_as_float((int)(gm >> 32)));
    }
}


// Per particle (sorted rank k): its leaf's centre-of-mass and quadrupole
// gradient terms added to its pair gradients, times G, written in input
// order.  With s = x - com (member offset from the leaf's centre of mass):
// d/dx += m (v + 6 S s - 2 tr(S) s), d/dm += g_M + v.s + 3 s.S s - tr(S) s.s.
__global__ void k_gleaf_out(const float4 *gl, const float4 *E0, const float4 *pw, const int32_t *pleaf,
                            double *gpart, const float4 *gpart32, int n, double G)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int i = pleaf[k];
        const float4 a = gl[3 * (size_t)i], b = gl[3 * (size_t)i + 1], c = gl[3 * (size_t)i + 2];
        const float v0 = a.x, v1 = a.y, v2 = a.z, tr = a.w;
        const float S0 = b.x, S1 = b.y, S2 = b.z, S3 = b.w, S4 = c.x, S5 = c.y;
        const double g0 = __longlong_as_double(((long long)__float_as_int(c.w) << 32) |
                                               (long long)(unsigned)__float_as_int(c.z));
        const float4 e = E0[i], x = pw[k];
        const float s0 = x.x - e.x, s1 = x.y - e.y, s2 = x.z - e.z;
        const float Ss0 = fmaf(S0, s0, fmaf(S3, s1, S4 * s2));
        const float Ss1 = fmaf(S3, s0, fmaf(S1, s1, S5 * s2));
        const float Ss2 = fmaf(S4, s0, fmaf(S5, s1, S2 * s2));
        const float ss = fmaf(s0, s0, fmaf(s1, s1, s2 * s2));
        const float sSs = fmaf(s0, Ss0, fmaf(s1, Ss1, s2 * Ss2));
        const float tm = fmaf(v0, s0, fmaf(v1, s1, fmaf(v2, s2, fmaf(3.f, sSs, -ss * tr))));
        const float m = x.w;
        const double2 p01 = *reinterpret_cast<const double2 *>(gpart + 4 * (size_t)k);
        const double2 p23 = *reinterpret_cast<const double2 *>(gpart + 4 * (size_t)k + 2);
        const float4 q = gpart32[k];
        double o0 = (p01.x + f64_of(q.x)) + f64_of(m * fmaf(6.f, Ss0, fmaf(-2.f * tr, s0, v0)));
        double o1 = (p01.y + f64_of(q.y)) + f64_of(m * fmaf(6.f, Ss1, fmaf(-2.f * tr, s1, v1)));
        double o2 = (p23.x + f64_of(q.z)) + f64_of(m * fmaf(6.f, Ss2, fmaf(-2.f * tr, s2, v2)));
        double o3 = (p23.y + f64_of(q.w)) + (g0 + f64_of(tm));
        if (G != 1.0) {
            o0 *= G;
            o1 *= G;
            o2 *= G;
            o3 *= G;
        }
        // in place, sorted order (coalesced); k_gather_out writes the input order
        *reinterpret_cast<double2 *>(gpart + 4 * (size_t)k) = make_double2(o0, o1);
        *reinterpret_cast<double2 *>(gpart + 4 * (size_t)k + 2) = make_double2(o2, o3);
    }
}

// Input-order outputs from the sorted per-particle results: a gather, so that
// the caller's arrays are written coalesced (scattered 24- and 8-byte writes
// into them cost partial-sector read-modify-writes).
__global__ void k_gather_out(const double *gsorted, const int32_t *rank, int n, double scale, double *d_pos,
                             double *d_mass)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const size_t k = (size_t)rank[i];
        const double2 a = *reinterpret_cast<const double2 *>(gsorted + 4 * k);
        const double2 b = *reinterpret_cast<const double2 *>(gsorted + 4 * k + 2);
        d_pos[3 * (size_t)i] = scale * a.x;
        d_pos[3 * (size_t)i + 1] = scale * a.y;
        d_pos[3 * (size_t)i + 2] = scale * b.x;
        d_mass[i] = scale * b.y;
    }
}

int accel_vjp(Tree *t, const int64_t *active, int64_t n_active, const double *cot_a, const double *cot_phi,
              double *d_pos, double *d_mass, cudaStream_t s)
{
    const int n = (int)t->n, nn = t->nn, BT = 256;
    Work w;
    WalkParams P;
    ph_begin(t, PH_VJP, s);
    // the forward's lists and groups when it was called with the same active set
    bool match = false;
    const bool lists = n_active > 0 && use_lists(t, s);
    if (lists) {
        int rc0 = lists_match(t, active, n_active, s, match);
        if (rc0) return rc0;
    }
    int rc = prepare(t, active, n_active, w, P, s, match && t->lists_grp_gen == t->grp_gen);
    if (rc) return rc;
    if (!t->lists_ok) match = false; // a new workspace: the list sizes were dropped with the old one
    // adjoint workspace: cotd [n][4] f64, cot [n] float4, gpart [n][4] f64, gnode [nn][10] f64,
    // gl [nn][3] float4, gpart32 [n][4] f32, gnode32 [nn][12] f32
    size_t need = align_up(32 * (size_t)n) + align_up(16 * (size_t)n) + align_up(32 * (size_t)n) +
                  align_up(80 * (size_t)nn) + align_up(48 * (size_t)nn) + align_up(16 * (size_t)n) +
                  align_up(48 * (size_t)nn);
    if (t->ws2_bytes < need) {
        // allocated while a stream is captured, the buffer would belong to the graph
        if (capturing(s)) return SFG_EINVAL;
        if (t->ws2) dev_free(t, t->ws2, s);
        t->ws2 = dev_alloc(t, need, s);
        if (!t->ws2) {
            t->ws2_bytes = 0;
            return SFG_ENOMEM;
        }
        t->ws2_bytes = need;
    }
    char *p = (char *)t->ws2;
    double *cotd = (double *)p;
    p += align_up(32 * (size_t)n);
    float4 *cot = (float4 *)p;
    p += align_up(16 * (size_t)n);
    double *gpart = (double *)p;
    p += align_up(32 * (size_t)n);
    double *gnode = (double *)p;
    p += align_up(80 * (size_t)nn);
    float4 *gl = (float4 *)p;
    p += align_up(48 * (size_t)nn);
    float *gpart32 = (float *)p;
    p += align_up(16 * (size_t)n);
    float *gnode32 = (float *)p;
    SFG_CUDA_OK(cudaMemsetAsync(cotd, 0, 32 * (size_t)n, s));
    SFG_CUDA_OK(cudaMemsetAsync(gpart, 0, 32 * (size_t)n, s));
    SFG_CUDA_OK(cudaMemsetAsync(gnode, 0, 80 * (size_t)nn, s));
    SFG_CUDA_OK(cudaMemsetAsync(gpart32, 0, 16 * (size_t)n, s));
    SFG_CUDA_OK(cudaMemsetAsync(gnode32, 0, 48 * (size_t)nn, s));
    if (n_active > 0) {
        k_cot_rows<<<grid_for(n_active, BT), BT, 0, s>>>(active, n_active, n, t->rank, w.pre, cot_a, cot_phi, cotd);
        k_cot_pack<<<grid_for(n, BT), BT, 0, s>>>(cotd, w.pre + n, cot);
        P.cot = cot;
        P.gpart = gpart;
        P.gnode = gnode;
        P.gpart32 = gpart32;
        P.gnode32 = gnode32;
        if (lists) {
            if (!match) {
                rc = build_lists(t, w, P, s, n_active);
                if (rc) return rc;
                rc = remember_active(t, active, n_active, s);
                if (rc) return rc;
            }
            items_from_counts(t, w, P, s, WT_VJP, true);
            rc = expand_lists(t, w, P, s);
            if (rc) return rc;
        } else {
            t->lists_ok = false;
            make_items(t, w, P, s);
        }
        if (t->timing) {
            int rc2 = cloud_timer_begin(t, 1, s, P);
            if (rc2) return rc2;
        }
        ph_begin(t, PH_VJP_WALK, s);
        if (lists) launch_eval<MODE_VJP>(t, P, s);
        else launch_walk<MODE_VJP>(t, P, s);
        ph_end(t, PH_VJP_WALK, s);
        k_gnode_unit<<<grid_for(nn, BT), BT, 0, s>>>(gnode, gnode32, t->nM, nn);
        t->n_launch += 4;
        // levels 1..top hold few nodes each: one block pushes them in one launch
        int top = 0;
        while (top + 1 <= t->depth && t->lvl_off[top + 2] - t->lvl_off[top + 1] <= 2048) top++;
        if (top >= 1) {
            PushLevels L;
            for (int l = 0; l < SFG_LMAX + 3; l++) L.off[l] = t->lvl_off[l];
            k_gnode_push_top<<<1, 256, 0, s>>>(gnode, t->ncom, t->nparent, L, top);
            t->n_launch += 1;
        }
        for (int l = top + 1; l <= t->depth; l++) {
            int b = t->lvl_off[l], e = t->lvl_off[l + 1];
            if (e > b) {
                k_gnode_push<<<grid_for(e - b, BT), BT, 0, s>>>(gnode, t->ncom, t->nparent, b, e);
                t->n_launch += 1;
            }
        }
        k_gleaf_prep<<<grid_for(nn, BT), BT, 0, s>>>(gnode, t->nnchild, nn, gl);
        k_gleaf_out<<<grid_for(n, BT), BT, 0, s>>>(gl, t->E0, t->pw, t->pleaf, gpart, (const float4 *)gpart32, n,
                                                   t->prm.G);
        k_gather_out<<<grid_for(n, BT), BT, 0, s>>>(gpart, t->rank, n, 1.0, d_pos, d_mass);
        t->n_launch += 2;
    } else {
        k_gather_out<<<grid_for(n, BT), BT, 0, s>>>(gpart, t->rank, n, t->prm.G, d_pos, d_mass);
    }
    t->n_launch += 1;
    ph_end(t, PH_VJP, s);
    SFG_CUDA_OK(cudaGetLastError());
    return SFG_OK;
}

int debug_lists(Tree *t, const int64_t *active, int64_t n_active, int64_t *n_groups, int64_t *n_p2m_total,
                int64_t *n_p2p_total, int64_t *groups, int32_t *p2m, int32_t *p2p, cudaStream_t s)
{
    Work w;
    WalkParams P;
    int rc = prepare(t, active, n_active, w, P, s);
    if (rc) return rc;
    int ng = 0;
    SFG_CUDA_OK(cudaMemcpyAsync(&ng, t->d_counters + 5, sizeof(int), cudaMemcpyDeviceToHost, s));
    SFG_CUDA_OK(cudaStreamSynchronize(s));
    int *cnt = (int *)dev_alloc(t, sizeof(int) * NCNT * (size_t)(ng > 0 ? ng : 1), s);
    if (!cnt) return SFG_ENOMEM;
    P.dbg_counts = cnt;
    launch_walk<MODE_COUNT>(t, P, s);
    int2 *gt_h = (int2 *)malloc(sizeof(int2) * (size_t)(ng > 0 ? ng : 1));
    int *cnt_h = (int *)malloc(sizeof(int) * NCNT * (size_t)(ng > 0 ? ng : 1));
    SFG_CUDA_OK(cudaMemcpyAsync(gt_h, w.gtab, sizeof(int2) * (size_t)ng, cudaMemcpyDeviceToHost, s));
    SFG_CUDA_OK(cudaMemcpyAsync(cnt_h, cnt, sizeof(int) * NCNT * (size_t)ng, cudaMemcpyDeviceToHost, s));
    SFG_CUDA_OK(cudaStreamSynchronize(s));
    long long tm = 0, tp = 0;
    long long *off_h = (long long *)malloc(sizeof(long long) * 2 * (size_t)(ng > 0 ? ng : 1));
    for (int g = 0; g < ng; g++) {
        off_h[2 * g] = tm;
        off_h[2 * g + 1] = tp;
        tm += cnt_h[NCNT * g];
        tp += cnt_h[NCNT * g + 1] + cnt_h[NCNT * g + 3];
    }
    *n_groups = ng;
    *n_p2m_total = tm;
    *n_p2p_total = tp;
    if (groups && p2m && p2p) {
        for (int g = 0; g < ng; g++) {
            groups[4 * g] = gt_h[g].x;
            groups[4 * g + 1] = gt_h[g].y;
            groups[4 * g + 2] = cnt_h[NCNT * g];
            groups[4 * g + 3] = cnt_h[NCNT * g + 1] + cnt_h[NCNT * g + 3];
        }
        long long *off_d = (long long *)dev_alloc(t, sizeof(long long) * 2 * (size_t)(ng > 0 ? ng : 1), s);
        int *dm = (int *)dev_alloc(t, sizeof(int) * (size_t)(tm > 0 ? tm : 1), s);
        int *dp = (int *)dev_alloc(t, sizeof(int) * (size_t)(tp > 0 ? tp : 1), s);
        if (!off_d || !dm || !dp) return SFG_ENOMEM;
        SFG_CUDA_OK(cudaMemcpyAsync(off_d, off_h, sizeof(long long) * 2 * (size_t)ng, cudaMemcpyHostToDevice, s));
        SFG_CUDA_OK(cudaMemsetAsync(t->d_counters + 2, 0, 3 * sizeof(unsigned long long), s));
        P.dbg_off = off_d;
        P.dbg_m = dm;
        P.dbg_p = dp;
        launch_walk<MODE_DUMP>(t, P, s);
        SFG_CUDA_OK(cudaMemcpyAsync(p2m, dm, sizeof(int) * (size_t)tm, cudaMemcpyDeviceToHost, s));
        SFG_CUDA_OK(cudaMemcpyAsync(p2p, dp, sizeof(int) * (size_t)tp, cudaMemcpyDeviceToHost, s));
        SFG_CUDA_OK(cudaStreamSynchronize(s));
        dev_free(t, off_d, s);
        dev_free(t, dm, s);
        dev_free(t, dp, s);
    }
    SFG_CUDA_OK(cudaStreamSynchronize(s));
    dev_free(t, cnt, s);
    free(gt_h);
    free(cnt_h);
    free(off_h);
    SFG_CUDA_OK(cudaGetLastError());
    return SFG_OK;
}

} // namespace sfg
