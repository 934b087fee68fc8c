// sfg_internal.cuh -- internal declarations of libsfg (not part of the ABI).
//
// Data layout in HBM (n particles, nn nodes; "sorted" = Morton order):
//   particles  key[n] u64, order[n] i32 (sorted rank -> original index),
//              rank[n] i32 (inverse), pos_s[n][3] f64, mass_s[n] f64,
//              soft_s[n] f64, sink_s[n] u8,
//              pw[n] float4 = (x - c_leaf (FP32), m),
//              pc[n] int4   = (leaf centre in half-cells (3 x i32), h bits; h < 0 for sinks)
//   nodes (breadth-first: ids ordered by (level, first sorted index); the
//   children of a node are consecutive ids)
//              nfirst/ncount/nparent/nchild_first/nnchild/nlevel [nn] i32
//              W0[nn] int4 = (lo.xyz, level | leaf << 8)       } walk record:
//              W1[nn] int4 = (hi.xyz, leaf ? first : child_first) } integer cell boxes,
//              W2[nn] int4 = (cq.xyz, leaf ? count : nchild)    } centre-of-mass cell
//              Whq[nn] u64 = ceil((h_max / cell)^2) capped at 2^62
//              E0[nn] float4 = (com - c_node (FP32), M)      } FP32 multipole record
//              E1[nn] float4 = (Qxx, Qyy, Qxy, Qxz)          } (Qzz = -Qxx - Qyy)
//              E2[nn] float4 = (Qyz, node centre in half-cells as 3 x i32 bits)
//              nM[nn], ncom[nn][3], nQ[nn][6], nhmax[nn] f64  } FP64 moments
// Grid: integer cells of side L0 / 2^21 from the frame origin x0; node and
// group centres are integers in half-cell units, so centre differences are
// exact in FP32 (|difference| < 2^22).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <unordered_set>
#include <vector>

#include "../../include/sfg.h"

#define SFG_LMAX 21
#define SFG_GRID_MAX 2097151u
#define SFG_CAP62 4611686018427387904ull

namespace sfg {

// status bits recorded on the device (mapped to SFG_E* on the host)
enum : int { ST_EINVAL = 1, ST_EOVERFLOW = 2, ST_ETIMEOUT = 4, ST_NODECAP = 8 };

struct Frame {
    double x0[3];
    double L0;
    double scale;     // 2^21 / L0 (exact)
    double half_cell; // L0 / 2^22 (exact)
};

constexpr int NCOUNTERS = 10;

struct Tree {
    sfg_params prm;
    int64_t n = 0;
    int nn = 0, cap = 0, depth = 0, n_levels = 0;
    int lvl_off[SFG_LMAX + 3] = {0};
    // a tree holds C >= 1 independent clouds (a forest): cloud c is the
    // particle range [off[c], off[c+1]) of the input and of the sorted order,
    // with its own frame and root (node c)
    int nclouds = 1;
    std::vector<int64_t> off_h;
    std::vector<Frame> frames_h;
    Frame frame_h{}; // frames_h[0]
    cudaStream_t stream = nullptr;
    int *d_status = nullptr;
    Frame *d_frame = nullptr; // [C]
    int64_t *d_off = nullptr; // [C + 1]
    unsigned long long *d_minmax = nullptr; // [C][6]
    int32_t *pcloud = nullptr;              // sorted rank -> cloud (C > 1)
    int32_t *ncloud = nullptr;              // node -> cloud
    int *d_lvl = nullptr; // device level offsets [SFG_LMAX + 3]
    // particles
    uint64_t *key = nullptr;
    int32_t *order = nullptr, *rank = nullptr;
    double *pos_s = nullptr, *mass_s = nullptr, *soft_s = nullptr;
    uint8_t *sink_s = nullptr;
    float4 *pw = nullptr;
    int4 *pc = nullptr;
    int32_t *pleaf = nullptr; // sorted rank -> its leaf
    // nodes
    int32_t *nfirst = nullptr, *ncount = nullptr, *nparent = nullptr, *nchild_first = nullptr,
            *nnchild = nullptr, *nlevel = nullptr;
    int4 *W0 = nullptr, *W1 = nullptr, *W2 = nullptr;
    unsigned long long *Whq = nullptr;
    float4 *E0 = nullptr, *E1 = nullptr, *E2 = nullptr;
    double *nM = nullptr, *ncom = nullptr, *nQ = nullptr, *nhmax = nullptr;
    // per-call workspace (grow-only)
    void *ws = nullptr, *ws2 = nullptr, *ws3 = nullptr, *ws4 = nullptr; // forward, adjoint, tidal, jerk
    size_t ws_bytes = 0, ws2_bytes = 0, ws3_bytes = 0, ws4_bytes = 0;
    sfg_stats last{};
    // [0] p2p, [1] p2m, [2] overflowed groups, [3] work, [4] retry work, [5] groups, [6] distinct targets,
    // [7] item cost total, [8] Newtonian-list P2P interactions
    unsigned long long *d_counters = nullptr;
    int *d_n = nullptr; // device copy of n
    long long n_launch = 0;
    bool timing = false;
    cudaEvent_t ev[10] = {};  // pairs: build, fwd, fwd walk, vjp, vjp walk
    bool ev_used[5] = {false, false, false, false, false};
    unsigned long long *d_ctime = nullptr; // [2][C + 1] per-cloud completion stamps (timing on)
    bool ctime_used[2] = {false, false};
    // stored interaction lists (store_lists): P2M node ids and P2P particle
    // ranges of every group of the active set they were walked for, kept for
    // the adjoint; the group table and list sizes stay in the workspace
    int *lm = nullptr;
    int2 *lr = nullptr;
    long long lm_cap = 0, lr_cap = 0;
    int *lp = nullptr; // the P2P ranges expanded to sorted particle ranks
    long long lp_cap = 0, lp_need = 0; // capacity; entries of the kept lists
    bool lp_ready = false;             // lp holds the kept lists' expansion
    int64_t *la = nullptr; // copy of that active index array
    int64_t la_cap = 0, la_n = -1;
    bool la_all = false;   // it was NULL (every particle)
    bool lists_ok = false;
    long long grp_gen = 0;        // groups formed so far (each call forms its active set's, unless reused)
    long long lists_grp_gen = -1; // grp_gen when the kept lists were built for the groups in the workspace
    // relative opening criterion: |g_prev| per sorted rank, alpha
    double *gps = nullptr;
    double rel_alpha = 0.0;
    bool rel_on = false;
    int *d_flag = nullptr;       // device scratch word
    long long *d_lscan = nullptr; // list-offset scan scratch + totals
    unsigned long long *d_lbump = nullptr; // one-pass list walk: reservations and flags
    void *lstage = nullptr;                // one-pass list walk: per-warp staging
    size_t lstage_bytes = 0;
    int list_walks = 0;                    // walks of the last stored-list build (1 or 2)
    // calls evaluate only the share of the groups of process share_rank of share_world
    int share_rank = 0, share_world = 1;
    std::unordered_set<void *> live; // every device allocation still held
};

// ---- memory ----
void *dev_alloc(Tree *t, size_t bytes, cudaStream_t s);
void dev_free(Tree *t, void *p, cudaStream_t s);

// ---- build (build.cu) ----
int build_tree(Tree *t, const double *pos, const double *mass, const double *soft, const uint8_t *is_sink,
               cudaStream_t s);

// ---- scans (build.cu) ----
// Exclusive scan of in[0..*d_n) into out[0..*d_n], out[*d_n] = total.  If
// extra_dst != NULL, *extra_dst = *extra_base + total.  max_n bounds *d_n.
// Scratch: scan_scratch_bytes() bytes.
size_t scan_scratch_bytes();
void scan_exclusive(const int *in, int *out, const int *d_n, int max_n, int *extra_dst, const int *extra_base,
                    void *scratch, cudaStream_t s);
// Single-pass form (one launch per scan) over a scratch of scan1p_bytes(max_n)
// bytes that init() zeroes once; the scan leaves it zeroed.  range() scans
// in[*d_lo .. *d_hi) (d_lo may be NULL: from 0) into out[0..len], out[len] =
// total, bounded by min(bound, max_n); a look-back wait that runs out sets
// ST_ETIMEOUT in *status.
size_t scan1p_bytes(int max_n);
struct Scan1P {
    unsigned *ctr = nullptr;            // [0] tile tickets, [1] blocks done
    unsigned long long *look = nullptr; // per tile: status (2 bits) | value (32 bits)
    int max_n = 0;
    void attach(void *mem, int max_n); // an already zeroed scratch
    void init(void *mem, int max_n, cudaStream_t s);
    void range(const int *in, int *out, const int *d_lo, const int *d_hi, int bound, int *extra_dst,
               const int *extra_base, int *status, cudaStream_t s) const;
    void exclusive(const int *in, int *out, const int *d_n, int bound, int *status, cudaStream_t s) const
    {
        range(in, out, nullptr, d_n, bound, nullptr, nullptr, status, s);
    }
};

// ---- forward / adjoint (walk.cu) ----
int accel(Tree *t, const int64_t *active, int64_t n_active, double *accel, double *phi, cudaStream_t s);
int accel_vjp(Tree *t, const int64_t *active, int64_t n_active, const double *cot_a, const double *cot_phi,
              double *d_pos, double *d_mass, cudaStream_t s);
int accel_tidal(Tree *t, const int64_t *active, int64_t n_active, double *accel, double *phi, double *tidal,
                cudaStream_t s);
int tidal_timestep(const double *tidal, int64_t n, double eta, double *dt, cudaStream_t s);
int set_relative(Tree *t, const double *g_prev, double alpha, cudaStream_t s);
int accel_jerk(Tree *t, const double *vel, const int64_t *active, int64_t n_active, double *accel, double *phi,
               double *jerk, cudaStream_t s);
int sink_timestep(Tree *t, const double *vel, const int64_t *active, int64_t n_active, double eta, double *dt,
                  cudaStream_t s);
int debug_lists(Tree *t, const int64_t *active, int64_t n_active, int64_t *n_groups, int64_t *n_p2m_total,
                int64_t *n_p2p_total, int64_t *groups, int32_t *p2m, int32_t *p2p, cudaStream_t s);

int num_sms();

// timing helpers (no-ops unless t->timing)
enum { PH_BUILD = 0, PH_FWD = 1, PH_FWD_WALK = 2, PH_VJP = 3, PH_VJP_WALK = 4 };
// Events recorded while a stream is being captured into a CUDA graph cannot
// be timed, so phase timing skips captured calls (the per-cloud completion
// stamps are written by the kernels and work in graphs too).
inline bool capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}
inline void ph_begin(Tree *t, int ph, cudaStream_t s)
{
    if (!t->timing) return;
    if (capturing(s)) {
        t->ev_used[ph] = false;
        return;
    }
    if (!t->ev[2 * ph]) {
        cudaEventCreate(&t->ev[2 * ph]);
        cudaEventCreate(&t->ev[2 * ph + 1]);
    }
    cudaEventRecord(t->ev[2 * ph], s);
}
inline void ph_end(Tree *t, int ph, cudaStream_t s)
{
    if (!t->timing || !t->ev[2 * ph] || capturing(s)) return;
    cudaEventRecord(t->ev[2 * ph + 1], s);
    t->ev_used[ph] = true;
}

// ---- device helpers ----
__host__ __device__ inline uint64_t spread3(uint32_t v)
{
    uint64_t x = v & 0x1fffffu;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

__host__ __device__ inline uint32_t compact3(uint64_t x)
{
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x1fffffull;
    return (uint32_t)x;
}

// Morton interleave: bit 3k+2 = x, 3k+1 = y, 3k = z.
__host__ __device__ inline uint64_t morton3(uint32_t qx, uint32_t qy, uint32_t qz)
{
    return (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
}

// Cell of coordinate x: floor((x - x0) scale) clamped to [0, 2^21 - 1].
// scale = 2^21 / L0 is a power of two, so the product is exact and its floor
// is read off the bits of the (rounded) difference with the exponent moved
// by log2(scale): one FP64 operation, the rest on the integer pipes.  A
// subnormal difference takes the FP64 product.
__device__ inline uint32_t cell_of(double x, double x0, double scale)
{
    const double t = __dsub_rn(x, x0);
    const long long tb = __double_as_longlong(t);
    if (tb <= 0) return 0u; // t <= 0 (the sign bit or +0)
    const int ex = (int)((tb >> 52) & 0x7ff);
    if (ex == 0x7ff) return (tb & 0xfffffffffffffll) ? 0u : SFG_GRID_MAX; // NaN: 0, +inf: clamped
    if (ex == 0) {
        const double s = __dmul_rn(t, scale);
        return s >= 2097152.0 ? SFG_GRID_MAX : (uint32_t)s;
    }
    const int se = (int)((__double_as_longlong(scale) >> 52) & 0x7ff) - 1023;
    const int e = ex - 1023 + se; // exponent of the product
    if (e < 0) return 0u;
    if (e >= 21) return SFG_GRID_MAX;
    const unsigned long long m = (unsigned long long)(tb & 0xfffffffffffffll) | (1ull << 52);
    return (uint32_t)(m >> (52 - e));
}

__device__ inline unsigned long long hq_of(double h, double scale)
{
    double v = __dmul_rn(h, scale);
    double v2 = __dmul_rn(v, v);
    if (!(v2 < 4611686018427387904.0)) return SFG_CAP62;
    unsigned long long c = (unsigned long long)ceil(v2);
    return c > 0 ? c : 1ull;
}

// The CUDA error behind the last SFG_ECUDA returned on this thread.
extern thread_local cudaError_t g_last_cuda_error;
inline int cuda_fail(cudaError_t e)
{
    g_last_cuda_error = e;
    return SFG_ECUDA;
}

#define SFG_CUDA_OK(expr)                                                                                    \
    do {                                                                                                     \
        cudaError_t _e = (expr);                                                                             \
        if (_e != cudaSuccess) return ::sfg::cuda_fail(_e);                                                  \
    } while (0)

} // namespace sfg
