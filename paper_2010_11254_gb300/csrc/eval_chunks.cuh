// eval_chunks.cuh -- forward and adjoint evaluation of stored interaction
// lists in source chunks (STARFORGE methods paper, Sec. 2.2 and 2.2.1);
// included by walk.cu, after the helpers it reuses (soft_KP, soft_KPR,
// ring_take, cp_async16, global_ns, WalkParams).
//
// One warp per work item.  The group's T targets are dealt two per lane:
// TL = ceil(T / 2) target lanes form a slice (8 for 13 or 14 targets),
// R = floor(32 / TL) slices, A = R TL active lanes, and lane (tl, s) holds
// targets tl and tl + TL.  Sources arrive in chunks of C = A CK_M (CK_M,
// the list depth, 1, 2 or 4): every active lane stages CK_M of them (P2M
// node ids, or sorted particle ranks of the group's expanded P2P list),
// converted to the group-centred FP32 frame (exact integer half-cell centre
// differences plus the stored FP32 offsets).  Slots past the end of a list
// hold massless sources far outside the cloud, so the pair loops run without
// bounds checks; each source read from shared memory serves two pairs.
//
// Forward: slice s evaluates the chunk's slots s, s + R, ...; potentials are
// summed in FP32 over a chunk and in float-float (two_sum_add) across
// chunks.  Adjoint: each slice takes blocks of TL consecutive slots; at step
// j lane tl pairs its targets with slot (tl + j) mod TL of the block, adds
// the source-side terms to an accumulator and hands it to lane tl - 1, so
// that after TL steps lane tl holds the sum over all targets for slot tl of
// the block and adds it to that source's FP32 gradient sum (P2P list entries
// are dealt to the blocks so that list neighbours land in different
// slices).  Pairs inside a softening support (possible on softened ranges
// only) are flagged and evaluated afterwards with the full pair rule, one
// per lane per round.
#pragma once

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

// Adds b to the float-float sum (hi, lo): the error-free two-sum of hi and b
// (Knuth's TwoSum, six FP32 additions) leaves hi + b = s + e exactly, e goes
// to lo.  hi + lo carries about 48 bits, as an FP64 accumulator of FP32 chunk
// sums would, at FP32 cost (FP64 arithmetic runs at 1/64 of the FP32 rate).
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float b)
{
    const float s = hi + b;
    const float v = s - hi;
    lo += (hi - (s - v)) + (b - v);
    hi = s;
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

// The evaluation at chunk depths 1, 2 and 4 (sfg_params.list_depth): a
// deeper chunk amortizes the per-chunk costs (waits, synchronizations,
// potential flushes) over more pairs and takes more shared memory per warp.
namespace ck1 {
constexpr int CK_M = 1;
#include "eval_chunks_body.inc"
} // namespace ck1
namespace ck2 {
constexpr int CK_M = 2;
#include "eval_chunks_body.inc"
} // namespace ck2
namespace ck4 {
constexpr int CK_M = 4;
#include "eval_chunks_body.inc"
} // namespace ck4
