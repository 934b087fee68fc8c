// eval_chunks.cuh -- forward and adjoint evaluation of stored interaction
// lists in source chunks (STARFORGE methods paper, Sec. 2.2 and 2.2.1);
// included by walk.cu, after the helpers it reuses (soft_KP, soft_KPR,
// ring_take, cp_async16, global_ns, WalkParams).
//
// One warp per work item.  The group's T targets are dealt two per lane:
// TL = ceil(T / 2) target lanes form a slice, R = floor(32 / TL) slices,
// A = R TL active lanes, and lane (tl, s) holds targets tl and tl + TL.
// Sources arrive in chunks of C = 2 A: every active lane stages two (P2M
// node ids, or sorted particle ranks of the group's expanded P2P list),
// converted to the group-centred FP32 frame (exact integer half-cell centre
// differences plus the stored FP32 offsets).  Slots past the end of a list
// hold massless sources far outside the cloud, so the pair loops run without
// bounds checks; each source read from shared memory serves two pairs.
//
// Forward: slice s evaluates the chunk's slots s, s + R, ...; potentials are
// summed in FP32 over a chunk and in FP64 across chunks.  Adjoint: each
// slice takes blocks of TL consecutive slots; at step j lane tl pairs its
// targets with slot (tl + j) mod TL of the block, adds the source-side
// terms to an accumulator and hands it to lane tl - 1, so that after TL
// steps lane tl holds the sum over all targets for slot tl of the block and
// adds it to that source's FP64 gradient.  Pairs inside a softening support
// (possible on softened ranges only) are flagged and evaluated afterwards
// with the full pair rule, one per lane per round.
#pragma once

constexpr int CK_M = 2;             // sources staged per active lane per chunk
constexpr int CK_MAX = 32 * CK_M;   // largest chunk
constexpr int CK_WARPS = 4;         // warps per block

struct ChunkSmem {
    float4 sA[CK_MAX];     // (x, y, z, m): group-centred position, mass
    float4 sB[CK_MAX];     // P2M: Qxx Qyy Qxy Qxz; softened P2P: h, 1/h, rank bits, sink flag
    float2 sC[CK_MAX];     // P2M: Qyz Qzz; softened P2P: h^2, -
    int sN[CK_MAX];        // source id (node id or sorted rank), -1 for padding
    float4 raw[3][CK_MAX]; // the next chunk's records in flight; reused for the slice sums at the end
    float4 sS[CK_MAX];     // adjoint: deferred pairs' source-side sums (dL/dx_j, dL/dm_j)
    float4 tI[32];         // targets: h, 1/h, rank bits, sink flag
};

// Source-side adjoint sums are added to FP32 gradient buffers with vector
// reductions (one 16- or 8-byte reduction for four or two values); every
// source of a list is visited once per group, so each entry sums one
// contribution per group that lists it (per particle, the groups whose P2P
// lists hold it; per node, the groups that accept it).  The buffers are added
// to the FP64 gradients before the node push-down.  Node gradients take 12
// floats per node: gM, gcom[3] | gQ xx yy zz xy | gQ xz yz, -, - .
constexpr int GN32 = 12;

__device__ __forceinline__ void red_add_v4(float *p, float a, float b, float c, float d)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

__device__ __forceinline__ void red_add_v2(float *p, float a, float b)
{
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}

// Lane layout and group frame of one work item.
struct ChunkGroup {
    int T, TL, R, A, tl, s, tfirst, cloud;
    int cg[3];       // group centre in half-cells
    float s22;       // half-cell size
    float far;       // 2 L0: padding sources sit at -far, absent targets at +far (every axis)
    bool active;     // lane < A
    int nxt;         // adjoint rotation: the lane this one reads its accumulator from
};

template <int NT>
struct ChunkTargets {
    float ox[NT], oy[NT], oz[NT];
    float ht2[NT];   // h^2 (0 for an absent target)
    unsigned valid;  // bit i: target i exists
};

constexpr int CK_NT = 2; // targets per lane

template <int NT>
__device__ __forceinline__ void chunk_setup(const WalkParams &P, ChunkSmem &S, int g, int lane, ChunkGroup &G,
                                            ChunkTargets<NT> &X)
{
    const int2 gt = P.gtab[g];
    G.tfirst = gt.x;
    G.T = gt.y;
    G.TL = (G.T + NT - 1) / NT;
    G.R = 32 / G.TL;
    G.A = G.R * G.TL;
    G.active = lane < G.A;
    G.tl = lane % G.TL;
    G.s = G.active ? lane / G.TL : 0;
    G.nxt = G.active ? G.s * G.TL + (G.tl + 1 == G.TL ? 0 : G.tl + 1) : lane;
    G.cloud = P.pcloud ? P.pcloud[P.tgt[G.tfirst]] : 0;
    const Frame fr = P.frames[G.cloud];
    G.s22 = (float)fr.half_cell;
    G.far = (float)(2.0 * fr.L0);
    uint32_t lo[3] = {SFG_GRID_MAX, SFG_GRID_MAX, SFG_GRID_MAX}, hi[3] = {0, 0, 0};
    int r[NT];
    X.valid = 0u;
#pragma unroll
    for (int i = 0; i < NT; i++) {
        const int t = G.tl + G.TL * i;
        r[i] = -1;
        if (G.active && t < G.T) {
            X.valid |= 1u << i;
            r[i] = P.tgt[G.tfirst + t];
            const uint64_t k = P.key[r[i]];
            const uint32_t q[3] = {compact3(k >> 2), compact3(k >> 1), compact3(k)};
#pragma unroll
            for (int a = 0; a < 3; a++) {
                lo[a] = min(lo[a], q[a]);
                hi[a] = max(hi[a], q[a]);
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int glo = (int)__reduce_min_sync(FULL, lo[a]);
        const int ghi = (int)__reduce_max_sync(FULL, hi[a]);
        G.cg[a] = glo + ghi + 1;
    }
    const double c0 = fr.x0[0] + (double)G.cg[0] * fr.half_cell;
    const double c1 = fr.x0[1] + (double)G.cg[1] * fr.half_cell;
    const double c2 = fr.x0[2] + (double)G.cg[2] * fr.half_cell;
#pragma unroll
    for (int i = 0; i < NT; i++) {
        if (X.valid >> i & 1u) {
            const double *x = P.pos_s + 3 * (size_t)r[i];
            const double h = P.soft_s[r[i]];
            const float hf = (float)h;
            X.ox[i] = (float)(x[0] - c0);
            X.oy[i] = (float)(x[1] - c1);
            X.oz[i] = (float)(x[2] - c2);
            X.ht2[i] = hf * hf;
            if (G.s == 0)
                S.tI[G.tl + G.TL * i] = make_float4(hf, 1.f / hf, __int_as_float(r[i]), P.sink_s[r[i]] ? 1.f : 0.f);
        } else {
            X.ox[i] = X.oy[i] = X.oz[i] = G.far;
            X.ht2[i] = 0.f;
        }
    }
}

// Padding slot: massless, far outside the cloud, no id; a node record with
// a zero quadrupole, a particle record of support 1 and rank -1.
template <bool NODE>
__device__ __forceinline__ void chunk_pad(ChunkSmem &S, int slot, float far)
{
    S.sA[slot] = make_float4(-far, -far, -far, 0.f);
    S.sB[slot] = NODE ? make_float4(0.f, 0.f, 0.f, 0.f) : make_float4(1.f, 1.f, __int_as_float(-1), 0.f);
    S.sC[slot] = make_float2(0.f, 0.f);
    S.sN[slot] = -1;
}

// ---- staging: P2M node records ----
__device__ __forceinline__ void chunk_fetch_nodes(const WalkParams &P, ChunkSmem &S, const ChunkGroup &G,
                                                  const int (&id)[CK_M], int lane)
{
    if (G.active) {
#pragma unroll
        for (int b = 0; b < CK_M; b++) {
            const int slot = lane + G.A * b;
            if ((unsigned)id[b] < (unsigned)P.nn) {
                cp_async16(&S.raw[0][slot], &P.E0[id[b]]);
                cp_async16(&S.raw[1][slot], &P.E1[id[b]]);
                cp_async16(&S.raw[2][slot], &P.E2[id[b]]);
            }
        }
    }
    cp_async_commit();
}

template <bool QUAD>
__device__ __forceinline__ void chunk_convert_nodes(const WalkParams &P, ChunkSmem &S, const ChunkGroup &G,
                                                    const int (&id)[CK_M], int lane)
{
    if (!G.active) return;
#pragma unroll
    for (int b = 0; b < CK_M; b++) {
        const int slot = lane + G.A * b;
        if ((unsigned)id[b] < (unsigned)P.nn) {
            const float4 e0 = S.raw[0][slot], e1 = S.raw[1][slot], e2 = S.raw[2][slot];
            const float px = fmaf((float)(__float_as_int(e2.y) - G.cg[0]), G.s22, e0.x);
            const float py = fmaf((float)(__float_as_int(e2.z) - G.cg[1]), G.s22, e0.y);
            const float pz = fmaf((float)(__float_as_int(e2.w) - G.cg[2]), G.s22, e0.z);
            S.sA[slot] = make_float4(px, py, pz, e0.w);
            if (QUAD) {
                S.sB[slot] = e1;
                S.sC[slot] = make_float2(e2.x, -(e1.x + e1.y));
            } else {
                S.sB[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
                S.sC[slot] = make_float2(0.f, 0.f);
            }
            S.sN[slot] = id[b];
        } else {
            if (id[b] != -1) atomicOr(P.status, ST_ETIMEOUT); // a corrupt list entry
            chunk_pad<true>(S, slot, G.far);
        }
    }
}

// ---- staging: P2P particle records (ranges queued in S.ring) ----
__device__ __forceinline__ void chunk_fetch_parts(const WalkParams &P, ChunkSmem &S, const ChunkGroup &G,
                                                  const int (&j)[CK_M], int lane)
{
    if (G.active) {
#pragma unroll
        for (int b = 0; b < CK_M; b++) {
            const int slot = lane + G.A * b;
            if (j[b] >= 0 && j[b] < P.npart) {
                cp_async16(&S.raw[0][slot], &P.pw[j[b]]);
                cp_async16(&S.raw[1][slot], &P.pc[j[b]]);
            }
        }
    }
    cp_async_commit();
}

template <bool SOFT>
__device__ __forceinline__ void chunk_convert_parts(const WalkParams &P, ChunkSmem &S, const ChunkGroup &G,
                                                    const int (&j)[CK_M], int lane)
{
    if (!G.active) return;
#pragma unroll
    for (int b = 0; b < CK_M; b++) {
        const int slot = lane + G.A * b;
        if (j[b] >= 0 && j[b] < P.npart) {
            const float4 a = S.raw[0][slot];
            const float4 c = S.raw[1][slot];
            const float px = fmaf((float)(__float_as_int(c.x) - G.cg[0]), G.s22, a.x);
            const float py = fmaf((float)(__float_as_int(c.y) - G.cg[1]), G.s22, a.y);
            const float pz = fmaf((float)(__float_as_int(c.z) - G.cg[2]), G.s22, a.z);
            S.sA[slot] = make_float4(px, py, pz, a.w);
            if (SOFT) {
                const float h = fabsf(c.w); // negative for a sink
                S.sB[slot] = make_float4(h, 1.f / h, __int_as_float(j[b]), c.w < 0.f ? 1.f : 0.f);
                S.sC[slot] = make_float2(h * h, 0.f);
            }
            S.sN[slot] = j[b];
        } else {
            if (j[b] != -1) atomicOr(P.status, ST_ETIMEOUT);
            chunk_pad<false>(S, slot, G.far);
        }
    }
}

// The item's share of a list of n entries cut in 32-entry tiles: [b, e).
__device__ __forceinline__ void item_share(int n, int kk, int K, int &b, int &e)
{
    const int nt = (n + 31) >> 5;
    const int t0 = (int)((long long)nt * kk / K), t1 = (int)((long long)nt * (kk + 1) / K);
    b = t0 * 32;
    e = min(n, t1 * 32);
    if (t0 >= t1) e = b;
}

// ------------------------------------------------------------- forward ----
// Monopole + quadrupole field of one node (Sec. 2.2): a = M d / r^3 - Q d / r^5
// + 5/2 (d.Qd) d / r^7, phi = -M / r - (d.Qd) / (2 r^5), d = com - x_i.
template <bool QUAD, int NT>
__device__ __forceinline__ void chunk_fwd_nodes(const ChunkSmem &S, const ChunkGroup &G, const ChunkTargets<NT> &X,
                                                float (&ax)[NT], float (&ay)[NT], float (&az)[NT], float (&pt)[NT])
{
    const int steps = G.TL * CK_M;
#pragma unroll(3 - NT)
    for (int i = 0; i < steps; i++) {
        const int k = i * G.R + G.s;
        const float4 p = S.sA[k];
        const float4 q = S.sB[k];
        const float2 q2 = S.sC[k]; // Qyz, Qzz
#pragma unroll
        for (int t = 0; t < NT; t++) {
            const float dx = p.x - X.ox[t], dy = p.y - X.oy[t], dz = p.z - X.oz[t];
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float rinv = rsqrtf(r2);
            const float ri2 = rinv * rinv;
            const float ri3 = ri2 * rinv;
            const float Mr3 = p.w * ri3;
            if (QUAD) {
                const float ri5 = ri3 * ri2;
                const float Qd0 = fmaf(q.x, dx, fmaf(q.z, dy, q.w * dz));
                const float Qd1 = fmaf(q.z, dx, fmaf(q.y, dy, q2.x * dz));
                const float Qd2 = fmaf(q.w, dx, fmaf(q2.x, dy, q2.y * dz));
                const float qr5 = fmaf(dx, Qd0, fmaf(dy, Qd1, dz * Qd2)) * ri5; // d.Qd / r^5
                const float c = fmaf(qr5, 2.5f * ri2, Mr3);
                ax[t] = fmaf(c, dx, fmaf(-ri5, Qd0, ax[t]));
                ay[t] = fmaf(c, dy, fmaf(-ri5, Qd1, ay[t]));
                az[t] = fmaf(c, dz, fmaf(-ri5, Qd2, az[t]));
                pt[t] = fmaf(-p.w, rinv, fmaf(-0.5f, qr5, pt[t]));
            } else {
                ax[t] = fmaf(Mr3, dx, ax[t]);
                ay[t] = fmaf(Mr3, dy, ay[t]);
                az[t] = fmaf(Mr3, dz, az[t]);
                pt[t] = fmaf(-p.w, rinv, pt[t]);
            }
        }
    }
}

// Newtonian pairs a = m d / r^3, phi = -m / r.  On a softened range a pair
// inside max(h_i, h_j) (the self pair included) is left out and flagged in
// mk[t] (bit = step) for the full pair rule.
template <bool SOFT, int NT>
__device__ __forceinline__ void chunk_fwd_parts(const ChunkSmem &S, const ChunkGroup &G, const ChunkTargets<NT> &X,
                                                float (&ax)[NT], float (&ay)[NT], float (&az)[NT], float (&pt)[NT],
                                                unsigned (&mk)[NT])
{
    const int steps = G.TL * CK_M;
    unsigned ib = 1u;
#pragma unroll(3 - NT)
    for (int i = 0; i < steps; i++, ib <<= 1) {
        const int k = i * G.R + G.s;
        const float4 p = S.sA[k];
        float hj2 = 0.f;
        if (SOFT) hj2 = S.sC[k].x;
#pragma unroll
        for (int t = 0; t < NT; t++) {
            const float dx = p.x - X.ox[t], dy = p.y - X.oy[t], dz = p.z - X.oz[t];
            float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            float m = p.w;
            if (SOFT) {
                const bool sft = r2 < fmaxf(X.ht2[t], hj2);
                if (sft) mk[t] |= ib;
                r2 = sft ? 1.f : r2;
                m = sft ? 0.f : m;
            }
            const float rinv = rsqrtf(r2);
            const float ri2 = rinv * rinv;
            const float mr3 = m * (ri2 * rinv);
            ax[t] = fmaf(mr3, dx, ax[t]);
            ay[t] = fmaf(mr3, dy, ay[t]);
            az[t] = fmaf(mr3, dz, az[t]);
            pt[t] = fmaf(-m, rinv, pt[t]);
        }
    }
}

// Softened pair (Sec. 2.2.1) of a target (its record ti, position o) and a
// staged source (p, hh): gas-gas averages the kernels of both supports, a
// pair with a sink takes one kernel of the larger support.  Returns the
// acceleration and potential terms (a, phi); zero for the self pair and
// padding.  Kept out of line: deferred pairs are rare, and the inner loops'
// code stays small.
__device__ __noinline__ float4 soft_pair_fwd(float4 ti, float ox, float oy, float oz, float4 p, float4 hh)
{
    if (__float_as_int(hh.z) == __float_as_int(ti.z) || __float_as_int(hh.z) < 0)
        return make_float4(0.f, 0.f, 0.f, 0.f);
    const float dx = p.x - ox, dy = p.y - oy, dz = p.z - oz;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const bool sink = ti.w != 0.f || hh.w != 0.f;
    const bool tbig = ti.x >= hh.x;
    const float ha = tbig ? ti.x : hh.x, hainv = tbig ? ti.y : hh.y;
    const float hb = sink ? ha : (tbig ? hh.x : ti.x), hbinv = sink ? hainv : (tbig ? hh.y : ti.y);
    const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
    const float r = r2 * rinv;
    float K1, P1, K2, P2;
    soft_KP(r, rinv, ha, hainv, K1, P1);
    soft_KP(r, rinv, hb, hbinv, K2, P2);
    const float mK = p.w * 0.5f * (K1 + K2);
    return make_float4(mK * dx, mK * dy, mK * dz, p.w * 0.5f * (P1 + P2));
}

// Adjoint of one softened pair: with the pair rule's K, P and R = dK/dr / r,
// l = m K c + m (R cd + cf K) d goes to the source (and -l to the target),
// and dL/dm_j = K cd + P cf.  Returns (l, dL/dm_j); zero for the self pair
// and padding.
__device__ __noinline__ float4 soft_pair_vjp(float4 ti, float ox, float oy, float oz, float4 c, float4 p, float4 hh)
{
    if (__float_as_int(hh.z) == __float_as_int(ti.z) || __float_as_int(hh.z) < 0)
        return make_float4(0.f, 0.f, 0.f, 0.f);
    const float dx = p.x - ox, dy = p.y - oy, dz = p.z - oz;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const bool sink = ti.w != 0.f || hh.w != 0.f;
    const bool tbig = ti.x >= hh.x;
    const float ha = tbig ? ti.x : hh.x, hainv = tbig ? ti.y : hh.y;
    const float hb = sink ? ha : (tbig ? hh.x : ti.x), hbinv = sink ? hainv : (tbig ? hh.y : ti.y);
    const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
    const float r = r2 * rinv;
    float K1, P1, R1, K2, P2, R2;
    soft_KPR(r, rinv, ha, hainv, K1, P1, R1);
    soft_KPR(r, rinv, hb, hbinv, K2, P2, R2);
    const float K = 0.5f * (K1 + K2), Pp = 0.5f * (P1 + P2), Rr = 0.5f * (R1 + R2);
    const float cd = fmaf(c.x, dx, fmaf(c.y, dy, c.z * dz));
    const float mK = p.w * K;
    const float sv = p.w * fmaf(Rr, cd, c.w * K);
    return make_float4(fmaf(mK, c.x, sv * dx), fmaf(mK, c.y, sv * dy), fmaf(mK, c.z, sv * dz), fmaf(K, cd, Pp * c.w));
}

template <int NT>
__device__ __forceinline__ void chunk_fwd_deferred(const ChunkSmem &S, const ChunkGroup &G, const ChunkTargets<NT> &X,
                                                   float (&ax)[NT], float (&ay)[NT], float (&az)[NT],
                                                   float (&pt)[NT], unsigned (&mk)[NT])
{
#pragma unroll
    for (int t = 0; t < NT; t++)
        if (!(X.valid >> t & 1u)) mk[t] = 0u;
    unsigned any = 0u;
#pragma unroll
    for (int t = 0; t < NT; t++) any |= mk[t];
    while (__any_sync(FULL, any != 0u)) {
        int t = -1, i = 0;
#pragma unroll
        for (int u = NT - 1; u >= 0; u--)
            if (mk[u]) t = u;
        if (t >= 0) {
            const unsigned m = t == 0 ? mk[0] : mk[NT - 1];
            i = __ffs(m) - 1;
            if (t == 0) mk[0] &= m - 1;
            else mk[NT - 1] &= m - 1;
            const int k = i * G.R + G.s;
            const float4 f = soft_pair_fwd(S.tI[G.tl + G.TL * t], t == 0 ? X.ox[0] : X.ox[NT - 1],
                                           t == 0 ? X.oy[0] : X.oy[NT - 1], t == 0 ? X.oz[0] : X.oz[NT - 1],
                                           S.sA[k], S.sB[k]);
            if (t == 0) {
                ax[0] += f.x;
                ay[0] += f.y;
                az[0] += f.z;
                pt[0] += f.w;
            } else {
                ax[NT - 1] += f.x;
                ay[NT - 1] += f.y;
                az[NT - 1] += f.z;
                pt[NT - 1] += f.w;
            }
        }
        any = 0u;
#pragma unroll
        for (int u = 0; u < NT; u++) any |= mk[u];
    }
}

// ------------------------------------------------------------- adjoint ----
// Node adjoint (see vjp_p2m_tile for the formulas): per pair the
// target side gets -gd, the node +gd (its centre of mass), dL/dM and dL/dQ
// (off-diagonal sums kept doubled, halved once before the atomics).
template <bool QUAD, int NT>
__device__ __forceinline__ void chunk_vjp_nodes(const WalkParams &P, const ChunkSmem &S, const ChunkGroup &G,
                                                const ChunkTargets<NT> &X, const float (&c0)[NT],
                                                const float (&c1)[NT], const float (&c2)[NT],
                                                const float (&cf)[NT], float (&gx)[NT], float (&gy)[NT],
                                                float (&gz)[NT], int lane)
{
    constexpr int NA = QUAD ? 10 : 4;
    for (int b = 0; b < CK_M; b++) {
        const int base = (G.s * CK_M + b) * G.TL;
        float acc[NA];
#pragma unroll
        for (int q = 0; q < NA; q++) acc[q] = 0.f;
        int kq = G.tl;
        for (int j = 0; j < G.TL; j++) {
            const int k = base + kq;
            kq = kq + 1 == G.TL ? 0 : kq + 1;
            const float4 p = S.sA[k];
            float4 qa = make_float4(0.f, 0.f, 0.f, 0.f);
            float2 qb = make_float2(0.f, 0.f);
            if (QUAD) {
                qa = S.sB[k]; // Qxx Qyy Qxy Qxz
                qb = S.sC[k]; // Qyz Qzz
            }
#pragma unroll
            for (int t = 0; t < NT; t++) {
                const float dx = p.x - X.ox[t], dy = p.y - X.oy[t], dz = p.z - X.oz[t];
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                const float rinv = rsqrtf(r2);
                const float ri2 = rinv * rinv, ri3 = ri2 * rinv;
                const float cd = fmaf(c0[t], dx, fmaf(c1[t], dy, c2[t] * dz));
                const float Mr3 = p.w * ri3;
                acc[0] = fmaf(cd, ri3, fmaf(-cf[t], rinv, acc[0]));
                float gd0, gd1, gd2;
                const float cdr2 = cd * ri2;
                if (QUAD) {
                    const float ri5 = ri3 * ri2, ri7 = ri5 * ri2;
                    const float Qd0 = fmaf(qa.x, dx, fmaf(qa.z, dy, qa.w * dz));
                    const float Qd1 = fmaf(qa.z, dx, fmaf(qa.y, dy, qb.x * dz));
                    const float Qd2 = fmaf(qa.w, dx, fmaf(qb.x, dy, qb.y * dz));
                    const float Qc0 = fmaf(qa.x, c0[t], fmaf(qa.z, c1[t], qa.w * c2[t]));
                    const float Qc1 = fmaf(qa.z, c0[t], fmaf(qa.y, c1[t], qb.x * c2[t]));
                    const float Qc2 = fmaf(qa.w, c0[t], fmaf(qb.x, c1[t], qb.y * c2[t]));
                    const float q = fmaf(dx, Qd0, fmaf(dy, Qd1, dz * Qd2));
                    const float cQd = fmaf(c0[t], Qd0, fmaf(c1[t], Qd1, c2[t] * Qd2));
                    const float kc = fmaf(2.5f * q, ri7, Mr3);
                    const float kq5 = ri5 * fmaf(5.f, cdr2, -cf[t]); // 5 cd / r^7 - cf / r^5
                    const float kd = fmaf(ri7, fmaf(q, fmaf(-17.5f, cdr2, 2.5f * cf[t]), 5.f * cQd),
                                          Mr3 * fmaf(-3.f, cdr2, cf[t]));
                    gd0 = fmaf(kc, c0[t], fmaf(-ri5, Qc0, fmaf(kq5, Qd0, kd * dx)));
                    gd1 = fmaf(kc, c1[t], fmaf(-ri5, Qc1, fmaf(kq5, Qd1, kd * dy)));
                    gd2 = fmaf(kc, c2[t], fmaf(-ri5, Qc2, fmaf(kq5, Qd2, kd * dz)));
                    const float sQ = 0.5f * kq5;
                    const float w0 = fmaf(sQ, dx, -ri5 * c0[t]), w1 = fmaf(sQ, dy, -ri5 * c1[t]),
                                w2 = fmaf(sQ, dz, -ri5 * c2[t]);
                    acc[4] = fmaf(w0, dx, acc[4]);
                    acc[5] = fmaf(w1, dy, acc[5]);
                    acc[6] = fmaf(w2, dz, acc[6]);
                    acc[7] = fmaf(w0, dy, fmaf(w1, dx, acc[7]));
                    acc[8] = fmaf(w0, dz, fmaf(w2, dx, acc[8]));
                    acc[9] = fmaf(w1, dz, fmaf(w2, dy, acc[9]));
                } else {
                    const float kd = Mr3 * fmaf(-3.f, cdr2, cf[t]);
                    gd0 = fmaf(Mr3, c0[t], kd * dx);
                    gd1 = fmaf(Mr3, c1[t], kd * dy);
                    gd2 = fmaf(Mr3, c2[t], kd * dz);
                }
                acc[1] += gd0;
                acc[2] += gd1;
                acc[3] += gd2;
                gx[t] -= gd0;
                gy[t] -= gd1;
                gz[t] -= gd2;
            }
#pragma unroll
            for (int q = 0; q < NA; q++) acc[q] = __shfl_sync(FULL, acc[q], G.nxt);
        }
        if (QUAD) {
            acc[7] *= 0.5f;
            acc[8] *= 0.5f;
            acc[9] *= 0.5f;
        }
        const int id = G.active ? S.sN[base + G.tl] : -1;
        if (id >= 0) {
            float *dst = P.gnode32 + GN32 * (size_t)id;
            red_add_v4(dst, acc[0], acc[1], acc[2], acc[3]);
            if (QUAD) {
                red_add_v4(dst + 4, acc[4 % NA], acc[5 % NA], acc[6 % NA], acc[7 % NA]);
                red_add_v2(dst + 8, acc[8 % NA], acc[9 % NA]);
            }
        }
    }
}

// Particle adjoint with the Newtonian kernel.  With l = m K c + m (R cd + cf K) d
// (K = 1/r^3, R = dK/dr / r = -3/r^5, cd = c.d) the source gets +l and
// dL/dm_j = K cd - cf / r, the target -l; the target's m K c part is summed
// as the scalar sK[t] and multiplied by c once per item.  On a softened
// range a pair inside max(h_i, h_j) is left out and flagged in mk[t] (bit =
// b TL + j).  The source sums of block b are left in a[b][0..3].
template <bool SOFT, int NT>
__device__ __forceinline__ void chunk_vjp_parts(const ChunkSmem &S, const ChunkGroup &G, const ChunkTargets<NT> &X,
                                                const float (&c0)[NT], const float (&c1)[NT],
                                                const float (&c2)[NT], const float (&cf)[NT], float (&gx)[NT],
                                                float (&gy)[NT], float (&gz)[NT], float (&sK)[NT],
                                                unsigned (&mk)[NT], float (&a)[CK_M][4])
{
    unsigned ib = 1u;
#pragma unroll
    for (int b = 0; b < CK_M; b++) {
        const int base = (G.s * CK_M + b) * G.TL;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, am = 0.f;
        int kq = G.tl;
        for (int j = 0; j < G.TL; j++, ib <<= 1) {
            const int k = base + kq;
            kq = kq + 1 == G.TL ? 0 : kq + 1;
            const float4 p = S.sA[k];
            float hj2 = 0.f;
            if (SOFT) hj2 = S.sC[k].x;
#pragma unroll
            for (int t = 0; t < NT; t++) {
                const float dx = p.x - X.ox[t], dy = p.y - X.oy[t], dz = p.z - X.oz[t];
                float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                bool sft = false;
                if (SOFT) {
                    sft = r2 < fmaxf(X.ht2[t], hj2);
                    if (sft) mk[t] |= ib;
                    r2 = sft ? 1.f : r2;
                }
                const float rinv = rsqrtf(r2);
                const float ri2 = rinv * rinv;
                float K = ri2 * rinv;
                float ri = rinv;
                if (SOFT) {
                    K = sft ? 0.f : K;
                    ri = sft ? 0.f : ri;
                }
                const float cd = fmaf(c0[t], dx, fmaf(c1[t], dy, c2[t] * dz));
                const float mK = p.w * K;
                const float sv = mK * fmaf(-3.f * ri2, cd, cf[t]);
                a0 = fmaf(mK, c0[t], fmaf(sv, dx, a0));
                a1 = fmaf(mK, c1[t], fmaf(sv, dy, a1));
                a2 = fmaf(mK, c2[t], fmaf(sv, dz, a2));
                am = fmaf(K, cd, fmaf(-ri, cf[t], am));
                sK[t] += mK;
                gx[t] = fmaf(-sv, dx, gx[t]);
                gy[t] = fmaf(-sv, dy, gy[t]);
                gz[t] = fmaf(-sv, dz, gz[t]);
            }
            a0 = __shfl_sync(FULL, a0, G.nxt);
            a1 = __shfl_sync(FULL, a1, G.nxt);
            a2 = __shfl_sync(FULL, a2, G.nxt);
            am = __shfl_sync(FULL, am, G.nxt);
        }
        a[b][0] = a0;
        a[b][1] = a1;
        a[b][2] = a2;
        a[b][3] = am;
    }
}

// Deferred softened pairs of the adjoint: target side into the lane's
// registers, source side into S.sS (shared-memory atomics), added to the
// lane's block sums afterwards.
template <int NT>
__device__ __forceinline__ void chunk_vjp_deferred(ChunkSmem &S, const ChunkGroup &G, const ChunkTargets<NT> &X,
                                                   const float (&c0)[NT], const float (&c1)[NT],
                                                   const float (&c2)[NT], const float (&cf)[NT], float (&gx)[NT],
                                                   float (&gy)[NT], float (&gz)[NT], unsigned (&mk)[NT],
                                                   float (&a)[CK_M][4], int lane)
{
    unsigned any = 0u;
#pragma unroll
    for (int t = 0; t < NT; t++) {
        if (!(X.valid >> t & 1u)) mk[t] = 0u;
        any |= mk[t];
    }
    if (!__any_sync(FULL, any != 0u)) return;
    if (G.active) {
#pragma unroll
        for (int b = 0; b < CK_M; b++) S.sS[lane + G.A * b] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncwarp();
    while (__any_sync(FULL, any != 0u)) {
        int t = -1;
#pragma unroll
        for (int u = NT - 1; u >= 0; u--)
            if (mk[u]) t = u;
        if (t >= 0) {
            const unsigned m = t == 0 ? mk[0] : mk[NT - 1];
            const int bit = __ffs(m) - 1;
            if (t == 0) mk[0] &= m - 1;
            else mk[NT - 1] &= m - 1;
            const int b = bit / G.TL, j = bit - b * G.TL;
            int kq = G.tl + j;
            if (kq >= G.TL) kq -= G.TL;
            const int k = (G.s * CK_M + b) * G.TL + kq;
            const float4 l = soft_pair_vjp(
                S.tI[G.tl + G.TL * t], t == 0 ? X.ox[0] : X.ox[NT - 1], t == 0 ? X.oy[0] : X.oy[NT - 1],
                t == 0 ? X.oz[0] : X.oz[NT - 1],
                t == 0 ? make_float4(c0[0], c1[0], c2[0], cf[0])
                       : make_float4(c0[NT - 1], c1[NT - 1], c2[NT - 1], cf[NT - 1]),
                S.sA[k], S.sB[k]);
            if (l.x != 0.f || l.y != 0.f || l.z != 0.f || l.w != 0.f) {
                atomicAdd(&S.sS[k].x, l.x);
                atomicAdd(&S.sS[k].y, l.y);
                atomicAdd(&S.sS[k].z, l.z);
                atomicAdd(&S.sS[k].w, l.w);
            }
            if (t == 0) {
                gx[0] -= l.x;
                gy[0] -= l.y;
                gz[0] -= l.z;
            } else {
                gx[NT - 1] -= l.x;
                gy[NT - 1] -= l.y;
                gz[NT - 1] -= l.z;
            }
        }
        any = 0u;
#pragma unroll
        for (int u = 0; u < NT; u++) any |= mk[u];
    }
    __syncwarp();
    if (G.active) {
#pragma unroll
        for (int b = 0; b < CK_M; b++) {
            const float4 v = S.sS[(G.s * CK_M + b) * G.TL + G.tl];
            a[b][0] += v.x;
            a[b][1] += v.y;
            a[b][2] += v.z;
            a[b][3] += v.w;
        }
    }
}

// The lane's block sums added to the gradients of the sources it holds.
__device__ __forceinline__ void chunk_vjp_flush(const WalkParams &P, const ChunkSmem &S, const ChunkGroup &G,
                                                const float (&a)[CK_M][4])
{
    if (!G.active) return;
#pragma unroll
    for (int b = 0; b < CK_M; b++) {
        const int id = S.sN[(G.s * CK_M + b) * G.TL + G.tl];
        if (id >= 0) red_add_v4(P.gpart32 + 4 * (size_t)id, a[b][0], a[b][1], a[b][2], a[b][3]);
    }
}

// ---------------------------------------------------------- one item ----
template <bool QUAD, int MODE, int NT>
__device__ __forceinline__ int chunk_item(const WalkParams &P, ChunkSmem &S, int g, int kk, int K, int lane)
{
    constexpr bool VJP = MODE == MODE_VJP;
    ChunkGroup G;
    ChunkTargets<NT> X;
    chunk_setup<NT>(P, S, g, lane, G, X);
    float ax[NT], ay[NT], az[NT], pt[NT], sK[NT];
    double ph[NT];
    float c0[NT], c1[NT], c2[NT], cf[NT];
#pragma unroll
    for (int i = 0; i < NT; i++) {
        ax[i] = ay[i] = az[i] = pt[i] = sK[i] = 0.f;
        ph[i] = 0.0;
        c0[i] = c1[i] = c2[i] = cf[i] = 0.f;
        if (VJP && (X.valid >> i & 1u)) {
            const float4 cv = P.cot[G.tfirst + G.tl + G.TL * i];
            c0[i] = cv.x;
            c1[i] = cv.y;
            c2[i] = cv.z;
            cf[i] = cv.w;
        }
    }
    __syncwarp();
    const int *cn = P.lcnt + NCNT * (size_t)g;
    const int nm = cn[0], nps = cn[2], npn = cn[4]; // P2M nodes, softened and Newtonian P2P particles
    const int C = G.A * CK_M;
    // ---- P2M: node ids one chunk ahead of their records, which run one chunk ahead of the evaluation
    {
        const int *lm = P.lm + P.lmo[g];
        int e0, e1;
        item_share(nm, kk, K, e0, e1);
        auto ids = [&](int cb, int (&id)[CK_M]) {
#pragma unroll
            for (int b = 0; b < CK_M; b++) {
                const int e = cb + lane + G.A * b;
                id[b] = (G.active && e < e1) ? lm[e] : -1;
            }
        };
        int idc[CK_M], idn[CK_M];
        if (e0 < e1) {
            ids(e0, idc);
            chunk_fetch_nodes(P, S, G, idc, lane);
            ids(e0 + C, idn);
        }
        for (int cb = e0; cb < e1; cb += C) {
            cp_async_wait();
            chunk_convert_nodes<QUAD>(P, S, G, idc, lane);
            __syncwarp();
            if (cb + C < e1) {
#pragma unroll
                for (int b = 0; b < CK_M; b++) idc[b] = idn[b];
                chunk_fetch_nodes(P, S, G, idc, lane);
                ids(cb + 2 * C, idn);
            }
            if (VJP) {
                chunk_vjp_nodes<QUAD, NT>(P, S, G, X, c0, c1, c2, cf, ax, ay, az, lane);
            } else {
                chunk_fwd_nodes<QUAD, NT>(S, G, X, ax, ay, az, pt);
#pragma unroll
                for (int i = 0; i < NT; i++) {
                    ph[i] += (double)pt[i];
                    pt[i] = 0.f;
                }
            }
            __syncwarp();
        }
    }
    // ---- P2P: the group's expanded list, softened particles then Newtonian ones;
    // ranks one chunk ahead of their records, which run one chunk ahead of the evaluation
    const long long lpo = P.lpo[g]; // < 0: the expansion had no room (reported on the status word)
    const int *lp = P.lp + (lpo < 0 ? 0 : lpo);
#pragma unroll 1
    for (int list = 0; list < (lpo < 0 ? 0 : 2); list++) {
        const bool soft = list == 0;
        const int *lq = soft ? lp : lp + nps;
        int e0, e1;
        item_share(soft ? nps : npn, kk, K, e0, e1);
        auto ranks = [&](int cb, int (&j)[CK_M]) {
#pragma unroll
            for (int b = 0; b < CK_M; b++) {
                const int e = cb + lane + G.A * b;
                j[b] = (G.active && e < e1) ? lq[e] : -1;
            }
        };
        int jc[CK_M], jn[CK_M];
        if (e0 < e1) {
            ranks(e0, jc);
            chunk_fetch_parts(P, S, G, jc, lane);
            ranks(e0 + C, jn);
        }
        for (int cb = e0; cb < e1; cb += C) {
            cp_async_wait();
            if (soft) chunk_convert_parts<true>(P, S, G, jc, lane);
            else chunk_convert_parts<false>(P, S, G, jc, lane);
            __syncwarp();
            if (cb + C < e1) {
#pragma unroll
                for (int b = 0; b < CK_M; b++) jc[b] = jn[b];
                chunk_fetch_parts(P, S, G, jc, lane);
                ranks(cb + 2 * C, jn);
            }
            unsigned mk[NT];
#pragma unroll
            for (int i = 0; i < NT; i++) mk[i] = 0u;
            if (VJP) {
                float a[CK_M][4];
                if (soft) {
                    chunk_vjp_parts<true, NT>(S, G, X, c0, c1, c2, cf, ax, ay, az, sK, mk, a);
                    chunk_vjp_deferred<NT>(S, G, X, c0, c1, c2, cf, ax, ay, az, mk, a, lane);
                } else {
                    chunk_vjp_parts<false, NT>(S, G, X, c0, c1, c2, cf, ax, ay, az, sK, mk, a);
                }
                chunk_vjp_flush(P, S, G, a);
            } else {
                if (soft) {
                    chunk_fwd_parts<true, NT>(S, G, X, ax, ay, az, pt, mk);
                    chunk_fwd_deferred<NT>(S, G, X, ax, ay, az, pt, mk);
                } else {
                    chunk_fwd_parts<false, NT>(S, G, X, ax, ay, az, pt, mk);
                }
#pragma unroll
                for (int i = 0; i < NT; i++) {
                    ph[i] += (double)pt[i];
                    pt[i] = 0.f;
                }
            }
            __syncwarp();
        }
    }
    // ---- per-target sums over the slices (in slice order), through shared memory
    if (VJP) {
#pragma unroll
        for (int i = 0; i < NT; i++) { // the target's m K c terms
            ax[i] = fmaf(-sK[i], c0[i], ax[i]);
            ay[i] = fmaf(-sK[i], c1[i], ay[i]);
            az[i] = fmaf(-sK[i], c2[i], az[i]);
        }
    }
    float4 *redA = S.raw[0];
    double *redP = (double *)S.raw[1];
    if (G.active) {
#pragma unroll
        for (int i = 0; i < NT; i++) {
            redA[lane * NT + i] = make_float4(ax[i], ay[i], az[i], 0.f);
            redP[lane * NT + i] = ph[i];
        }
    }
    __syncwarp();
    float rx = 0.f, ry = 0.f, rz = 0.f;
    double rp = 0.0;
    const bool own = lane < G.T;
    if (own) {
        const int tl = lane % G.TL, ti = lane / G.TL;
        for (int s = 0; s < G.R; s++) {
            const int e = (s * G.TL + tl) * NT + ti;
            const float4 v = redA[e];
            rx += v.x;
            ry += v.y;
            rz += v.z;
            rp += redP[e];
        }
    }
    if (VJP) {
        if (own) {
            double *dst = P.gpart + 4 * (size_t)P.tgt[G.tfirst + lane];
            atomicAdd(dst, (double)rx);
            atomicAdd(dst + 1, (double)ry);
            atomicAdd(dst + 2, (double)rz);
        }
    } else if (K == 1) {
        if (own) {
            P.res_a[G.tfirst + lane] = make_float4(rx, ry, rz, 0.f);
            P.res_phi[G.tfirst + lane] = rp;
        }
    } else {
        // partial sums of this item; the group's last item sums them in k order
        const size_t slot = (size_t)(P.soff[g] + kk) * 32;
        if (own) {
            P.part_a[slot + lane] = make_float4(rx, ry, rz, 0.f);
            P.part_phi[slot + lane] = rp;
        }
        __threadfence();
        __syncwarp();
        int last = 0;
        if (lane == 0) last = atomicAdd(&P.gdone[g], 1) == K - 1;
        last = __shfl_sync(FULL, last, 0);
        if (last) {
            __threadfence();
            if (own) {
                float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
                double p = 0.0;
                const size_t s0 = (size_t)P.soff[g] * 32;
                for (int k = 0; k < K; k++) {
                    const float4 v = __ldcg(&P.part_a[s0 + (size_t)k * 32 + lane]);
                    a.x += v.x;
                    a.y += v.y;
                    a.z += v.z;
                    p += __ldcg(&P.part_phi[s0 + (size_t)k * 32 + lane]);
                }
                P.res_a[G.tfirst + lane] = a;
                P.res_phi[G.tfirst + lane] = p;
            }
        }
    }
    if (lane == 0 && kk == 0) {
        // count the group's list once (self pairs excluded)
        const unsigned long long T = (unsigned long long)G.T;
        atomicAdd(&P.counters[0], T * (unsigned long long)(nps + npn - 1));
        atomicAdd(&P.counters[1], T * (unsigned long long)nm);
        if (npn) atomicAdd(&P.counters[8], T * (unsigned long long)npn);
    }
    __syncwarp(); // the slice sums are read before the next item stages into raw
    return G.cloud;
}

// Persistent warps take work items (longest first) from an atomic counter.
// resident blocks per SM the register budget must allow: the adjoint keeps
// more per-lane state (cotangents, source sums) than the forward
constexpr int chunk_minb(int mode) { return mode == MODE_VJP ? 4 : 5; }

template <bool QUAD, int MODE>
__global__ void __launch_bounds__(CK_WARPS * 32, chunk_minb(MODE)) k_eval_chunks(WalkParams P)
{
    __shared__ ChunkSmem sm[CK_WARPS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    ChunkSmem &S = sm[w];
    const int nwork = P.ioff[*P.d_ngroups];
    if (P.ctime && lane == 0) atomicMin(&P.ctime[P.nclouds], global_ns());
    while (true) {
        int w_i = 0;
        if (lane == 0) w_i = (int)atomicAdd(&P.counters[3], 1ull);
        w_i = __shfl_sync(FULL, w_i, 0);
        if (w_i >= nwork) break;
        const int2 it = P.items[w_i];
        const int cloud = chunk_item<QUAD, MODE, CK_NT>(P, S, it.x, it.y, P.kcnt[it.x], lane);
        if (P.ctime && lane == 0) atomicMax(&P.ctime[cloud], global_ns());
    }
}
