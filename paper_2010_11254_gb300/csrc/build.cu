// build.cu -- tree construction on the GPU (STARFORGE methods paper, Sec. 2.2:
// the oct-tree that recursively subdivides the domain; node multipoles).
//
// Steps (one CUDA stream, all device-side; sfg_build synchronizes once):
//   1. validate inputs and reduce per-axis min/max (FP64 values compared as
//      order-preserving 64-bit integers: exact and order-free);
//   2. frame: origin x0 = per-axis minimum, root side L0 = smallest power of
//      two >= the largest extent;
//   3. keys: cell q = floor((x - x0) 2^21 / L0) per axis (clamped), 63-bit
//      Morton key, value = original index;
//   4. stable LSD radix sort of (key, index), 8 passes of 8 bits: every
//      pass's digit counts in one read of the keys, then one launch per pass
//      (tile offsets by a bounded decoupled look-back);
//   5. gather sorted FP64 particle arrays;
//   6. octree, one level at a time: a node with > N_leaf particles below
//      level 21 is split into its non-empty octants (binary search of the
//      child digit in the node's sorted key range); node ids are breadth-first;
//   7. moments, bottom-up: leaves sum their members in sorted order (one
//      lane per leaf, leaves taken by member count; on large clouds from
//      chunks staged in shared memory), then the internal levels, deepest
//      first, combine their children in octant order (parallel-axis
//      theorem; one launch per level, the small top levels in one block).
//      The operation order is fixed and this file is compiled without FMA
//      contraction, so the FP64 moments are reproducible bit for bit.
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "sfg_internal.cuh"

namespace sfg {

// ---------------------------------------------------------------- scans ----
constexpr int SCAN_NB = 512;
constexpr int SCAN_BT = 256;

__device__ inline int warp_incl_scan(int v)
{
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Inclusive block scan; returns the block total in *total.  Uses sh[32].
__device__ inline int block_incl_scan(int v, int *sh, int *total)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = warp_incl_scan(v);
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = lane < nw ? sh[lane] : 0;
        s = warp_incl_scan(s);
        if (lane < nw) sh[lane] = s;
    }
    __syncthreads();
    int pre = w > 0 ? sh[w - 1] : 0;
    *total = sh[nw - 1];
    __syncthreads();
    return x + pre;
}

// Length of the scanned range [lo, min(hi, max_n)): entries at max_n and
// beyond were never written (a level of the octree clamped to the node
// capacity), so they are not read.
__device__ inline int scan_len(const int *d_lo, const int *d_hi, int max_n)
{
    int lo = d_lo ? *d_lo : 0;
    int hi = min(*d_hi, max_n);
    return hi > lo ? hi - lo : 0;
}

__global__ void k_scan_reduce(const int *in, const int *d_lo, const int *d_hi, int max_n, int *bsum)
{
    __shared__ int sh[32];
    int n = scan_len(d_lo, d_hi, max_n);
    int chunk = (n + SCAN_NB - 1) / SCAN_NB;
    int b0 = min(n, blockIdx.x * chunk), b1 = min(n, b0 + chunk);
    int s = 0;
    for (int i = b0 + threadIdx.x; i < b1; i += blockDim.x) s += in[i];
    int tot;
    block_incl_scan(s, sh, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_top(int *bsum, const int *d_lo, const int *d_hi, int max_n, int *out, int *extra_dst,
                           const int *extra_base)
{
    __shared__ int sh[32];
    int v = bsum[threadIdx.x];
    int tot;
    int incl = block_incl_scan(v, sh, &tot);
    bsum[threadIdx.x] = incl - v;
    if (threadIdx.x == 0) {
        int n = scan_len(d_lo, d_hi, max_n);
        out[n] = tot;
        if (extra_dst) *extra_dst = (int)min((long long)*extra_base + tot, (long long)INT_MAX);
    }
}

__global__ void k_scan_down(const int *in, int *out, const int *d_lo, const int *d_hi, int max_n, const int *bsum)
{
    __shared__ int sh[32];
    int n = scan_len(d_lo, d_hi, max_n);
    int chunk = (n + SCAN_NB - 1) / SCAN_NB;
    int b0 = min(n, blockIdx.x * chunk), b1 = min(n, b0 + chunk);
    int carry = bsum[blockIdx.x];
    for (int base = b0; base < b1; base += blockDim.x) {
        int i = base + threadIdx.x;
        int v = i < b1 ? in[i] : 0;
        int tot;
        int incl = block_incl_scan(v, sh, &tot);
        if (i < b1) out[i] = carry + incl - v;
        carry += tot;
    }
}

size_t scan_scratch_bytes() { return SCAN_NB * sizeof(int); }

// Range-length form: n = *d_hi - *d_lo (d_lo may be NULL).
static void scan_range(const int *in, int *out, const int *d_lo, const int *d_hi, int max_n, int *extra_dst,
                       const int *extra_base, void *scratch, cudaStream_t s)
{
    // three launches
    int *bsum = (int *)scratch;
    k_scan_reduce<<<SCAN_NB, SCAN_BT, 0, s>>>(in, d_lo, d_hi, max_n, bsum);
    k_scan_top<<<1, SCAN_NB, 0, s>>>(bsum, d_lo, d_hi, max_n, out, extra_dst, extra_base);
    k_scan_down<<<SCAN_NB, SCAN_BT, 0, s>>>(in, out, d_lo, d_hi, max_n, bsum);
}

void scan_exclusive(const int *in, int *out, const int *d_n, int max_n, int *extra_dst, const int *extra_base,
                    void *scratch, cudaStream_t s)
{
    scan_range(in, out, nullptr, d_n, max_n, extra_dst, extra_base, scratch, s);
}

// Single-pass exclusive scan (one launch): tiles of SP_TILE entries taken
// in ticket order by a persistent grid; a tile publishes its total, then
// its inclusive prefix once the tiles before it are known (decoupled
// look-back, waits bounded: ST_ETIMEOUT).  The last block out zeroes the
// tickets and look-back words, so the scratch is zero between scans and is
// cleared once, when allocated.
constexpr int SP_BT = 256, SP_ITEMS = 8, SP_TILE = SP_BT * SP_ITEMS;
constexpr unsigned long long SP_AGG = 1ull << 62, SP_INC = 2ull << 62, SP_VAL = 0xffffffffull;

static int sp_tiles(int max_n) { return std::max(1, (max_n + SP_TILE - 1) / SP_TILE); }

size_t scan1p_bytes(int max_n) { return 16 + 8 * (size_t)sp_tiles(max_n); }

__global__ void __launch_bounds__(SP_BT)
    k_scan_1p(const int *in, int *out, const int *d_lo, const int *d_hi, int max_n, int *extra_dst,
              const int *extra_base, unsigned *ctr, unsigned long long *look, int *status)
{
    __shared__ int sh[32];
    __shared__ int s_tile, s_pre;
    __shared__ bool s_last;
    const int n = scan_len(d_lo, d_hi, max_n);
    const int ntiles = max(1, (n + SP_TILE - 1) / SP_TILE);
    for (;;) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(&ctr[0], 1u);
        __syncthreads();
        const int tile = s_tile;
        if (tile >= ntiles) break;
        const int i0 = tile * SP_TILE + threadIdx.x * SP_ITEMS;
        int v[SP_ITEMS], sum = 0;
#pragma unroll
        for (int k = 0; k < SP_ITEMS; k++) {
            v[k] = i0 + k < n ? in[i0 + k] : 0;
            sum += v[k];
        }
        int tot;
        const int incl = block_incl_scan(sum, sh, &tot);
        if (threadIdx.x == 0) {
            unsigned pre = 0;
            if (tile > 0) {
                atomicExch(&look[tile], SP_AGG | (unsigned)tot);
                for (long long j = tile - 1, spin = 0; j >= 0;) {
                    const unsigned long long x = *(volatile unsigned long long *)(look + j);
                    const unsigned long long f = x & ~SP_VAL;
                    if (f == 0ull) {
                        if (++spin > (1ll << 24)) { // a tile that never published: give up
                            atomicOr(status, ST_ETIMEOUT);
                            break;
                        }
                        continue;
                    }
                    pre += (unsigned)(x & SP_VAL);
                    if (f == SP_INC) break;
                    j--;
                }
            }
            atomicExch(&look[tile], SP_INC | (pre + (unsigned)tot));
            s_pre = (int)pre;
            if (tile == ntiles - 1) {
                const int total = (int)pre + tot;
                out[n] = total;
                if (extra_dst) *extra_dst = (int)min((long long)*extra_base + total, (long long)INT_MAX);
            }
        }
        __syncthreads();
        int run = s_pre + incl - sum;
#pragma unroll
        for (int k = 0; k < SP_ITEMS; k++) {
            if (i0 + k < n) out[i0 + k] = run;
            run += v[k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) s_last = atomicAdd(&ctr[1], 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last) {
        for (int t = threadIdx.x; t < ntiles; t += blockDim.x) look[t] = 0ull;
        if (threadIdx.x == 0) {
            ctr[0] = 0u;
            ctr[1] = 0u;
        }
    }
}

void Scan1P::attach(void *mem, int max_n_)
{
    ctr = (unsigned *)mem;
    look = (unsigned long long *)((char *)mem + 16);
    max_n = max_n_;
}

void Scan1P::init(void *mem, int max_n_, cudaStream_t s)
{
    attach(mem, max_n_);
    cudaMemsetAsync(mem, 0, scan1p_bytes(max_n), s);
}

void Scan1P::range(const int *in, int *out, const int *d_lo, const int *d_hi, int bound, int *extra_dst,
                   const int *extra_base, int *status, cudaStream_t s) const
{
    const int grid = std::min(sp_tiles(std::min(bound, max_n)), 2 * num_sms());
    k_scan_1p<<<grid, SP_BT, 0, s>>>(in, out, d_lo, d_hi, std::min(bound, max_n), extra_dst, extra_base, ctr, look,
                                     status);
}

// Depth of the last tree built in this process: the octree enqueues that
// many levels before its first look at the level sizes.
static std::atomic<int> g_depth_hint{SFG_LMAX};

int num_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

__global__ void k_set_int(int *p, int v) { *p = v; }

// ------------------------------------------------------ validate + frame ----
__device__ inline unsigned long long ord_of(double x)
{
    long long b = __double_as_longlong(x);
    return b >= 0 ? (unsigned long long)b ^ 0x8000000000000000ull : ~(unsigned long long)b;
}
__device__ inline double from_ord(unsigned long long u)
{
    long long b = (u & 0x8000000000000000ull) ? (long long)(u ^ 0x8000000000000000ull) : (long long)~u;
    return __longlong_as_double(b);
}

__global__ void k_minmax_init(unsigned long long *mm, int C)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 6 * C; i += gridDim.x * blockDim.x)
        mm[i] = (i % 6) < 3 ? ~0ull : 0ull;
}

// Grid (chunks, C): block (x, c) strides over cloud c's range only.
__global__ void k_validate_minmax(const double *pos, const double *mass, const double *soft, const int64_t *off,
                                  unsigned long long *mm_all, int *status)
{
    const int c = blockIdx.y;
    const int b = (int)off[c], e = (int)off[c + 1];
    unsigned long long *mm = mm_all + 6 * (size_t)c;
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0, 0, 0};
    bool bad = false;
    // checks on the bit patterns (the FP64 pipe is slow on this part):
    // finite = exponent field below all ones; m >= 0 = sign clear or -0; h > 0
    // = sign clear and not +0
    constexpr unsigned long long EXP = 0x7ff0000000000000ull, SIGN = 0x8000000000000000ull;
    for (int i = b + blockIdx.x * blockDim.x + threadIdx.x; i < e; i += gridDim.x * blockDim.x) {
        for (int a = 0; a < 3; a++) {
            double x = pos[3 * (size_t)i + a];
            if ((__double_as_longlong(x) & EXP) == EXP) bad = true;
            unsigned long long u = ord_of(x);
            lo[a] = u < lo[a] ? u : lo[a];
            hi[a] = u > hi[a] ? u : hi[a];
        }
        const unsigned long long mb = (unsigned long long)__double_as_longlong(mass[i]);
        const unsigned long long hb = (unsigned long long)__double_as_longlong(soft[i]);
        if ((mb & EXP) == EXP || ((mb & SIGN) && mb != SIGN)) bad = true;
        if ((hb & EXP) == EXP || (hb & SIGN) || hb == 0ull) bad = true;
    }
    for (int a = 0; a < 3; a++) {
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo[a], o);
            unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hi[a], o);
            lo[a] = l2 < lo[a] ? l2 : lo[a];
            hi[a] = h2 > hi[a] ? h2 : hi[a];
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&mm[a], lo[a]);
            atomicMax(&mm[3 + a], hi[a]);
        }
    }
    if (bad) atomicOr(status, ST_EINVAL);
}

__global__ void k_frame(const unsigned long long *mm_all, Frame *fr_all, int C, int *status)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const unsigned long long *mm = mm_all + 6 * (size_t)c;
    Frame *fr = fr_all + c;
    double E = 0.0;
    for (int a = 0; a < 3; a++) {
        double lo = from_ord(mm[a]), hi = from_ord(mm[3 + a]);
        fr->x0[a] = lo;
        double e = hi - lo;
        if (e > E) E = e;
    }
    double L0;
    if (E == 0.0) {
        L0 = 1.0;
    } else {
        long long b = __double_as_longlong(E);
        int ex = (int)((b >> 52) & 0x7ff);
        long long mant = b & 0xfffffffffffffll;
        if (ex == 0 || ex >= 0x7fe) {
            atomicOr(status, ST_EINVAL); // subnormal or huge extent: outside the supported domain
            L0 = 1.0;
        } else {
            L0 = mant == 0 ? E : ldexp(1.0, ex - 1023 + 1);
        }
    }
    fr->L0 = L0;
    fr->scale = ldexp(1.0, SFG_LMAX) / L0;
    fr->half_cell = ldexp(L0, -22);
}

// ------------------------------------------------------------------ keys ----
// Grid (chunks, C); also records the cloud of every input particle.
__global__ void k_keys(const double *pos, const int64_t *off, const Frame *frames, uint64_t *key, uint32_t *val,
                       uint16_t *cloud_of)
{
    const int c = blockIdx.y;
    const int b = (int)off[c], e = (int)off[c + 1];
    const Frame *fr = frames + c;
    const double x0 = fr->x0[0], y0 = fr->x0[1], z0 = fr->x0[2], sc = fr->scale;
    for (int i = b + blockIdx.x * blockDim.x + threadIdx.x; i < e; i += gridDim.x * blockDim.x) {
        if (cloud_of) cloud_of[i] = (uint16_t)c;
        uint32_t qx = cell_of(pos[3 * (size_t)i], x0, sc);
        uint32_t qy = cell_of(pos[3 * (size_t)i + 1], y0, sc);
        uint32_t qz = cell_of(pos[3 * (size_t)i + 2], z0, sc);
        key[i] = morton3(qx, qy, qz);
        val[i] = (uint32_t)i;
    }
}

// ------------------------------------------------------------ radix sort ----
constexpr int RS_WARPS = 8;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_WARPS * 32 * RS_ITEMS; // 4096

// Digit of element (k, v): 8 key bits at `shift`, or, with a cloud table,
// 8 bits of the cloud id of value v.
__device__ __forceinline__ int rs_digit(uint64_t k, uint32_t v, int shift, const uint16_t *cl)
{
    return cl ? (int)((cl[v] >> shift) & 255) : (int)((k >> shift) & 255);
}

__global__ void __launch_bounds__(RS_WARPS * 32)
    k_rs_hist(const uint64_t *key, const uint32_t *val, int n, int shift, int *hist, int nb, const uint16_t *cl)
{
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int base = blockIdx.x * RS_TILE, end = min(n, base + RS_TILE);
    for (int i = base + threadIdx.x; i < end; i += blockDim.x) atomicAdd(&h[rs_digit(key[i], val[i], shift, cl)], 1);
    __syncthreads();
    hist[threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_WARPS * 32)
    k_rs_scatter(const uint64_t *kin, const uint32_t *vin, uint64_t *kout, uint32_t *vout, int n, int shift,
                 const int *off, int nb, const uint16_t *cl)
{
    __shared__ int wcnt[RS_WARPS][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = lane; d < 256; d += 32) wcnt[w][d] = 0;
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
    uint64_t k[RS_ITEMS];
    uint32_t v[RS_ITEMS];
    int dg[RS_ITEMS], loc[RS_ITEMS];
    int base = blockIdx.x * RS_TILE + w * 32 * RS_ITEMS;
#pragma unroll
    for (int r = 0; r < RS_ITEMS; r++) {
        int i = base + r * 32 + lane;
        bool valid = i < n;
        k[r] = valid ? kin[i] : 0;
        v[r] = valid ? vin[i] : 0;
        int d = valid ? rs_digit(k[r], v[r], shift, cl) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int before = __popc(peers & lt);
        int c0 = valid ? wcnt[w][d] : 0;
        __syncwarp();
        if (valid && (31 - __clz(peers)) == lane) wcnt[w][d] = c0 + __popc(peers);
        __syncwarp();
        dg[r] = d;
        loc[r] = c0 + before;
    }
    __syncthreads();
    // per digit: exclusive prefix over warps (thread t owns digit t)
    {
        int d = threadIdx.x;
        int run = 0;
        for (int ww = 0; ww < RS_WARPS; ww++) {
            int c = wcnt[ww][d];
            wcnt[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ITEMS; r++) {
        if (dg[r] < 256) {
            int p = off[dg[r] * nb + blockIdx.x] + wcnt[w][dg[r]] + loc[r];
            kout[p] = k[r];
            vout[p] = v[r];
        }
    }
}


// ----------------------------------------------------- one-sweep passes ----
// Each pass of the stable LSD sort in one launch: the global count of every
// digit of every pass is taken once up front (it does not depend on the
// order), and each tile finds its offsets per digit by a decoupled look-back
// over the tiles before it.  Tiles are numbered in the order blocks start
// (an atomic counter), so every tile a block waits on has started and never
// waits on a later one; the waits are bounded all the same and give up with
// ST_ETIMEOUT.
constexpr int RS_MAXPASS = 10;                     // 8 key passes + up to 2 cloud-id passes
constexpr int OS_ITEMS = 8;                        // keys per thread of a one-sweep tile
constexpr int OS_TILE = RS_WARPS * 32 * OS_ITEMS;  // 2048 keys: few registers, 4 blocks per SM
constexpr unsigned long long RS_AGG = 1ull << 32;  // look-back word: flag in the high half, count below
constexpr unsigned long long RS_INC = 2ull << 32;
constexpr int LB_W = 4; // look-back words read per round

__global__ void __launch_bounds__(256)
    k_rs_count_all(const uint64_t *key, int n, const uint16_t *cloud_of, int cloud_passes, unsigned *gcount)
{
    __shared__ unsigned h[RS_MAXPASS][256];
    for (int i = threadIdx.x; i < RS_MAXPASS * 256; i += blockDim.x) (&h[0][0])[i] = 0u;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint64_t k = key[i];
#pragma unroll
        for (int p = 0; p < 8; p++) atomicAdd(&h[p][(k >> (8 * p)) & 255], 1u);
        if (cloud_passes) {
            const unsigned c = cloud_of[i]; // the values are the input indices at this point
            for (int q = 0; q < cloud_passes; q++) atomicAdd(&h[8 + q][(c >> (8 * q)) & 255], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < (8 + cloud_passes) * 256; i += blockDim.x) {
        const unsigned v = (&h[0][0])[i];
        if (v) atomicAdd(&gcount[i], v);
    }
}

// Exclusive prefix of the digit counts of each pass (one block of 256).
__global__ void k_rs_start(const unsigned *gcount, int npass, unsigned *gstart)
{
    __shared__ unsigned sh[256];
    for (int p = 0; p < npass; p++) {
        sh[threadIdx.x] = gcount[p * 256 + threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned run = 0;
            for (int d = 0; d < 256; d++) {
                const unsigned c = sh[d];
                sh[d] = run;
                run += c;
            }
        }
        __syncthreads();
        gstart[p * 256 + threadIdx.x] = sh[threadIdx.x];
        __syncthreads();
    }
}

// The lanes holding the same 8-bit digit d as this one (valid lanes only; the
// invalid lanes form their own set), from one ballot per digit bit: cheaper
// here than one __match_any_sync (build on 2e7 particles 6.42 -> 6.33 ms).
__device__ __forceinline__ unsigned digit_peers(int d, bool valid)
{
    const unsigned vm = __ballot_sync(0xffffffffu, valid);
    unsigned peers = valid ? vm : ~vm;
#pragma unroll
    for (int b = 0; b < 8; b++) {
        const unsigned bb = __ballot_sync(0xffffffffu, (d >> b) & 1);
        peers &= ((d >> b) & 1) ? bb : ~bb;
    }
    return peers;
}

__global__ void __launch_bounds__(RS_WARPS * 32, 4)
    k_rs_onesweep(const uint64_t *kin, const uint32_t *vin, uint64_t *kout, uint32_t *vout, int n, int shift,
                  const uint16_t *cl, const unsigned *gstart, unsigned long long *look, unsigned *tile_ctr,
                  int *status)
{
    __shared__ int wcnt[RS_WARPS][256];
    __shared__ unsigned start[256]; // global rank of the tile's first key of each digit
    __shared__ int toff[256];       // tile rank of the tile's first key of each digit
    __shared__ int sh[32];
    __shared__ int s_tile;
    // the tile reordered by digit, then written out in digit runs (coalesced)
    __shared__ uint64_t sk[OS_TILE];
    __shared__ uint32_t sv[OS_TILE];
    __shared__ uint8_t sd[OS_TILE];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(tile_ctr, 1u);
    for (int d = lane; d < 256; d += 32) wcnt[w][d] = 0;
    __syncthreads();
    const int tile = s_tile;
    const unsigned lt = (1u << lane) - 1u;
    uint64_t k[OS_ITEMS];
    uint32_t v[OS_ITEMS];
    int dg[OS_ITEMS], loc[OS_ITEMS];
    const int base = tile * OS_TILE + w * 32 * OS_ITEMS;
    // all of the thread's loads in flight before the first digit is ranked
#pragma unroll
    for (int r = 0; r < OS_ITEMS; r++) {
        const int i = base + r * 32 + lane;
        k[r] = i < n ? kin[i] : 0;
        v[r] = i < n ? vin[i] : 0;
    }
#pragma unroll
    for (int r = 0; r < OS_ITEMS; r++) {
        const bool valid = base + r * 32 + lane < n;
        int d = valid ? rs_digit(k[r], v[r], shift, cl) : 256;
        const unsigned peers = digit_peers(d, valid);
        int before = __popc(peers & lt);
        int c0 = valid ? wcnt[w][d] : 0;
        __syncwarp();
        if (valid && (31 - __clz(peers)) == lane) wcnt[w][d] = c0 + __popc(peers);
        __syncwarp();
        dg[r] = d;
        loc[r] = c0 + before;
    }
    __syncthreads();
    {
        // thread t owns digit t: exclusive prefix over the warps, the tile's
        // count, its offset in the tile, then the count of all earlier tiles
        // by look-back
        const int d = threadIdx.x;
        unsigned run = 0;
        for (int ww = 0; ww < RS_WARPS; ww++) {
            const int c = wcnt[ww][d];
            wcnt[ww][d] = (int)run;
            run += (unsigned)c;
        }
        int tot;
        toff[d] = block_incl_scan((int)run, sh, &tot) - (int)run;
        unsigned long long *mine = look + (size_t)tile * 256 + d;
        unsigned excl = 0;
        if (tile == 0) {
            atomicExch(mine, RS_INC | run);
        } else {
            atomicExch(mine, RS_AGG | run);
            // Look-back over LB_W predecessors per round, their words read
            // together: the tiles of the first wave all start at once, and a
            // tile there finds an inclusive prefix only about tile / 2 tiles
            // back, so a one-word-per-round walk would chain that many L2
            // round trips.  Published words are consumed in order up to the
            // first inclusive one (the end) or the first unpublished one (read
            // again next round).
            int j = tile - 1;
            for (long long spin = 0; j >= 0;) {
                unsigned long long x[LB_W];
#pragma unroll
                for (int q = 0; q < LB_W; q++)
                    x[q] = j - q >= 0 ? *(volatile unsigned long long *)(look + (size_t)(j - q) * 256 + d) : +RS_INC;
                int used = 0;
                bool end = false;
#pragma unroll
                for (int q = 0; q < LB_W; q++) {
                    if (end || used < q) continue;
                    const unsigned long long f = x[q] & ~0xffffffffull;
                    if (f == 0ull) continue; // unpublished: stop consuming here
                    excl += (unsigned)x[q];
                    used = q + 1;
                    end = f == RS_INC;
                }
                if (end) break;
                if (used == 0 && ++spin > (1ll << 24)) { // a tile that never published: give up
                    atomicOr(status, ST_ETIMEOUT);
                    break;
                }
                j -= used;
            }
            atomicExch(mine, RS_INC | (excl + run));
        }
        start[d] = gstart[d] + excl;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < OS_ITEMS; r++) {
        if (dg[r] < 256) {
            const int p = toff[dg[r]] + wcnt[w][dg[r]] + loc[r];
            sk[p] = k[r];
            sv[p] = v[r];
            sd[p] = (uint8_t)dg[r];
        }
    }
    __syncthreads();
    const int cnt = min(OS_TILE, n - tile * OS_TILE);
    for (int q = threadIdx.x; q < cnt; q += RS_WARPS * 32) {
        const int d = sd[q];
        const unsigned p = start[d] + (unsigned)(q - toff[d]);
        kout[p] = sk[q];
        vout[p] = sv[q];
    }
}

// --------------------------------------------------------------- gather ----
constexpr int PK_UNROLL = 4;
__global__ void k_pack(const double *pos, const double *mass, const double *soft, const uint8_t *sink, int n,
                       const uint32_t *val, int32_t *order, int32_t *rank, double *pos_s, double *mass_s,
                       double *soft_s, uint8_t *sink_s, const uint16_t *cloud_of, int32_t *pcloud)
{
    // PK_UNROLL ranks per thread and round, so that their gathers are in
    // flight together
    const int stride = gridDim.x * blockDim.x;
    for (int r0 = blockIdx.x * blockDim.x + threadIdx.x; r0 < n; r0 += PK_UNROLL * stride) {
        int idx[PK_UNROLL];
#pragma unroll
        for (int u = 0; u < PK_UNROLL; u++) {
            const int r = r0 + u * stride;
            idx[u] = r < n ? (int)val[r] : -1;
        }
        double x[PK_UNROLL][3], m[PK_UNROLL], h[PK_UNROLL];
        uint8_t sk[PK_UNROLL];
        uint16_t cl[PK_UNROLL];
#pragma unroll
        for (int u = 0; u < PK_UNROLL; u++) {
            const int i = idx[u] < 0 ? 0 : idx[u];
            if (idx[u] >= 0) {
                for (int a = 0; a < 3; a++) x[u][a] = pos[3 * (size_t)i + a];
                m[u] = mass[i];
                h[u] = soft[i];
                sk[u] = sink ? (uint8_t)(sink[i] != 0) : (uint8_t)0;
                cl[u] = pcloud ? cloud_of[i] : (uint16_t)0;
            }
        }
#pragma unroll
        for (int u = 0; u < PK_UNROLL; u++) {
            const int r = r0 + u * stride, i = idx[u];
            if (i < 0) continue;
            if (pcloud) pcloud[r] = cl[u];
            order[r] = i;
            rank[i] = r;
            for (int a = 0; a < 3; a++) pos_s[3 * (size_t)r + a] = x[u][a];
            mass_s[r] = m[u];
            soft_s[r] = h[u];
            sink_s[r] = sk[u];
        }
    }
}

// --------------------------------------------------------------- octree ----
// Every KS-th sorted key, so that the child boundaries of a large node are
// first bracketed in this small, cache-resident array and then searched in a
// window of at most KS keys, instead of by long strides through the keys.
constexpr int KS_LOG = 8, KS = 1 << KS_LOG;

__global__ void k_key_samples(const uint64_t *key, int n, uint64_t *ks)
{
    const int ns = (n + KS - 1) >> KS_LOG;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ns; j += gridDim.x * blockDim.x)
        ks[j] = key[(size_t)j << KS_LOG];
}

// Child boundaries of the node [f, e) at child shift cshift: s[d] = first
// index whose child digit is >= d (s[0] = f, s[8] = e; digits are
// non-decreasing inside the node).  The seven searches run in lockstep so
// their loads overlap; a node longer than a few sample strides is bracketed
// on the samples first.
__device__ inline void digit_bounds(const uint64_t *key, const uint64_t *ks, int f, int e, int cshift, int s[9])
{
    int lo[7], hi[7];
    const int k0 = (f + KS - 1) >> KS_LOG, k1 = (e - 1) >> KS_LOG; // samples inside [f, e): k0..k1
    if (k1 - k0 >= 4) {
        // first sample k in [k0, k1 + 1) with digit >= d
#pragma unroll
        for (int d = 0; d < 7; d++) {
            lo[d] = k0;
            hi[d] = k1 + 1;
        }
        for (int it = 0; it < 32 && (1 << it) <= k1 + 1 - k0; it++) {
#pragma unroll
            for (int d = 0; d < 7; d++) {
                if (lo[d] < hi[d]) {
                    int mid = (lo[d] + hi[d]) >> 1;
                    if (((ks[mid] >> cshift) & 7u) < (uint32_t)(d + 1)) lo[d] = mid + 1;
                    else hi[d] = mid;
                }
            }
        }
        // the boundary lies after sample k - 1 and at or before sample k
#pragma unroll
        for (int d = 0; d < 7; d++) {
            const int k = lo[d];
            lo[d] = k == k0 ? f : ((k - 1) << KS_LOG) + 1;
            hi[d] = k > k1 ? e : (k << KS_LOG);
        }
    } else {
#pragma unroll
        for (int d = 0; d < 7; d++) {
            lo[d] = f;
            hi[d] = e;
        }
    }
    int n = 0;
#pragma unroll
    for (int d = 0; d < 7; d++) n = max(n, hi[d] - lo[d]);
    for (int it = 0; it < 32 && (1 << it) <= n; it++) {
#pragma unroll
        for (int d = 0; d < 7; d++) {
            if (lo[d] < hi[d]) {
                int mid = (lo[d] + hi[d]) >> 1;
                if (((key[mid] >> cshift) & 7u) < (uint32_t)(d + 1)) lo[d] = mid + 1;
                else hi[d] = mid;
            }
        }
    }
    s[0] = f;
#pragma unroll
    for (int d = 0; d < 7; d++) s[d + 1] = lo[d];
    s[8] = e;
}

// One root per cloud: node c covers cloud c's sorted range.
__global__ void k_oct_root(const int64_t *off, int C, int32_t *nfirst, int32_t *ncount, int32_t *nparent,
                           int32_t *nlevel, int32_t *ncloud, int *lvl)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        nfirst[c] = (int)off[c];
        ncount[c] = (int)(off[c + 1] - off[c]);
        nparent[c] = -1;
        nlevel[c] = 0;
        ncloud[c] = c;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        lvl[0] = 0;
        lvl[1] = C;
    }
}

// Child boundaries of a large node [f, e) found by the whole block: every
// round, PROBE threads per digit read keys spread evenly over that digit's
// remaining interval, so each interval shrinks about PROBE + 1-fold per
// dependent load instead of 2-fold.  Invariant: the answer for digit d (first
// index with child digit >= d + 1) lies in [lo[d], hi[d]], and is hi[d] when
// no index of [lo[d], hi[d]) qualifies.  Every thread of the block calls it.
constexpr int BIG_NODE = 4096;

__device__ void block_digit_bounds(const uint64_t *key, int f, int e, int cshift, int *lo, int *hi, int *first)
{
    const int PROBE = blockDim.x / 7;
    const int tid = threadIdx.x, d = tid / PROBE, j = tid - d * PROBE;
    if (tid < 7) {
        lo[tid] = f;
        hi[tid] = e;
    }
    __syncthreads();
    for (int round = 0; round < 32; round++) {
        bool open = false;
#pragma unroll
        for (int q = 0; q < 7; q++) open |= lo[q] < hi[q];
        if (!open) break; // uniform: every thread reads the same shared values
        if (tid < 7) first[tid] = PROBE;
        __syncthreads();
        int pos = -1;
        if (d < 7 && lo[d] < hi[d]) {
            const int len = hi[d] - lo[d];
            pos = len <= PROBE ? (j < len ? lo[d] + j : -1)
                               : lo[d] + (int)(((long long)(j + 1) * len) / (PROBE + 1));
            if (pos >= 0 && ((key[pos] >> cshift) & 7u) >= (uint32_t)(d + 1)) atomicMin(&first[d], j);
        }
        __syncthreads();
        if (tid < 7 && lo[tid] < hi[tid]) {
            const int len = hi[tid] - lo[tid], k = first[tid];
            if (len <= PROBE) {
                const int a = k < len ? lo[tid] + k : hi[tid];
                lo[tid] = hi[tid] = a;
            } else {
                const int qk = lo[tid] + (int)(((long long)(k + 1) * len) / (PROBE + 1));
                const int qp = lo[tid] + (int)(((long long)k * len) / (PROBE + 1)); // probe k - 1 (k > 0)
                const int nlo = k == 0 ? lo[tid] : qp + 1;
                const int nhi = k < PROBE ? qk : hi[tid];
                lo[tid] = nlo;
                hi[tid] = nhi;
            }
        }
        __syncthreads();
    }
}

// Child counts of the level's nodes (tmp) and their child boundaries s[1..7]
// (bnd, 7 per node, read back by k_oct_write instead of searching again).
// Nodes longer than BIG_NODE are searched by a whole block each, the others
// by one thread each.
__global__ void k_oct_count(const uint64_t *key, const uint64_t *ks, const int *lvl, int level, int leaf_size, int cap,
                            const int32_t *nfirst, const int32_t *ncount, int *tmp, int *bnd, int *status)
{
    __shared__ int s_lo[7], s_hi[7], s_first[7];
    int b = lvl[level], e = lvl[level + 1];
    if (e > cap) {
        e = cap;
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, ST_NODECAP);
    }
    // block searches only on levels with few nodes (the top of the tree, where
    // the nodes are long); elsewhere every node goes to the thread path
    const bool blocks = level < SFG_LMAX && e - b <= 2 * (int)gridDim.x;
    if (blocks) {
        for (int node = b + blockIdx.x; node < e; node += gridDim.x) {
            const int c = ncount[node];
            if (c <= BIG_NODE || c <= leaf_size) continue;
            const int f = nfirst[node];
            block_digit_bounds(key, f, f + c, 3 * (SFG_LMAX - level - 1), s_lo, s_hi, s_first);
            if (threadIdx.x == 0) {
                int nch = 0, prev = f;
                for (int q = 0; q < 7; q++) {
                    nch += s_lo[q] > prev;
                    prev = s_lo[q];
                    bnd[7 * (size_t)(node - b) + q] = s_lo[q];
                }
                nch += f + c > prev;
                tmp[node - b] = nch;
            }
            __syncthreads();
        }
    }
    for (int node = b + blockIdx.x * blockDim.x + threadIdx.x; node < e; node += gridDim.x * blockDim.x) {
        int f = nfirst[node], c = ncount[node];
        if (blocks && c > BIG_NODE && c > leaf_size) continue; // done by a block above
        int nch = 0;
        if (c > leaf_size && level < SFG_LMAX) {
            int sb[9];
            digit_bounds(key, ks, f, f + c, 3 * (SFG_LMAX - level - 1), sb);
#pragma unroll
            for (int d = 0; d < 8; d++) nch += sb[d + 1] > sb[d];
#pragma unroll
            for (int d = 1; d < 8; d++) bnd[7 * (size_t)(node - b) + d - 1] = sb[d];
        }
        tmp[node - b] = nch;
    }
}

__global__ void k_oct_write(const int *bnd, const int *lvl, int level, int leaf_size, int cap, int32_t *nfirst,
                            int32_t *ncount, int32_t *nparent, int32_t *nchild_first, int32_t *nnchild,
                            int32_t *nlevel, int32_t *ncloud, const int *tmp_off, int *status)
{
    int b = lvl[level], e = min(lvl[level + 1], cap);
    int next = lvl[level + 1];
    for (int node = b + blockIdx.x * blockDim.x + threadIdx.x; node < e; node += gridDim.x * blockDim.x) {
        int f = nfirst[node], c = ncount[node];
        if (!(c > leaf_size && level < SFG_LMAX)) {
            nchild_first[node] = -1;
            nnchild[node] = 0;
            continue;
        }
        int cf = next + tmp_off[node - b];
        int sb[9];
        sb[0] = f;
#pragma unroll
        for (int d = 1; d < 8; d++) sb[d] = bnd[7 * (size_t)(node - b) + d - 1];
        sb[8] = f + c;
        int k = 0;
        const int cl = ncloud[node];
        for (int d = 0; d < 8; d++) {
            if (sb[d + 1] > sb[d]) {
                int id = cf + k;
                if (id < cap) {
                    nfirst[id] = sb[d];
                    ncount[id] = sb[d + 1] - sb[d];
                    nparent[id] = node;
                    nlevel[id] = level + 1;
                    ncloud[id] = cl;
                } else {
                    atomicOr(status, ST_NODECAP);
                }
                k++;
            }
        }
        nchild_first[node] = cf;
        nnchild[node] = k;
    }
}

// -------------------------------------------------------------- moments ----
struct MomArgs {
    const uint64_t *key;
    const double *pos, *mass, *soft;
    const uint8_t *sink;
    const int32_t *nfirst, *ncount, *nparent, *nchild_first, *nnchild, *nlevel, *ncloud;
    const Frame *fr; // [C]
    int4 *W0, *W1, *W2;
    unsigned long long *Whq;
    float4 *E0, *E1, *E2;
    double *nM, *ncom, *nQ, *nhmax;
    double *nS; // [nn][6] second moment about the centre of mass (scratch of the reduction)
    float4 *pw;
    int4 *pc;
    int32_t *pleaf;
    int nn;
};

__device__ inline void node_centre(const Frame &fr, const uint32_t lo[3], int level, int ci[3], double c[3])
{
    int sh = SFG_LMAX - level;
    for (int a = 0; a < 3; a++) {
        uint32_t corner = (lo[a] >> sh) << sh;
        ci[a] = (int)(2u * corner + (1u << sh));
        c[a] = fr.x0[a] + (double)(2u * corner + (1u << sh)) * fr.half_cell;
    }
}

// IEEE 754 round-to-nearest-even conversion FP64 -> FP32 on the integer
// pipes (FP64 operations, conversions included, issue at 1/64 of the FP32
// rate on this part, and the moment passes are bound by them).  A value in
// the normal FP32 exponent range keeps the top 23 of its 52 fraction bits;
// the 29 bits below decide the rounding (above half: up; exactly half: to
// even); a carry out of the fraction moves into the exponent, up to infinity
// past the largest float.  The rest (zeros, FP32-subnormal magnitudes,
// values past the FP32 range, infinities, NaN) goes to f32_rn_rare, out of
// line so that no FP64 conversion is issued on the common path.
__device__ __noinline__ unsigned f32_rn_rare(unsigned long long b)
{
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int E = (int)((b >> 52) & 0x7ffu);
    const unsigned long long frac = b & ((1ull << 52) - 1);
    if (E == 0x7ff) return sign | 0x7f800000u | (frac ? 0x400000u : 0u); // infinity; NaN made quiet
    const int e = E - 1023;
    if (e > 127) return sign | 0x7f800000u; // past the largest float: infinity
    if (E == 0) return sign;                // zero and FP64 subnormals round to zero
    // |x| < 2^-126: the FP32 subnormal q 2^-149 with q = RNE(mant 2^(e + 97)), a
    // right shift by s = -(e + 97) >= 30 of the 53-bit significand
    const unsigned long long mant = frac | (1ull << 52);
    const int sh = -(e + 97);
    if (sh > 54) return sign; // below half the smallest subnormal
    const unsigned long long q = mant >> sh, rem = mant & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    return sign | (unsigned)(q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull));
}

__device__ __forceinline__ float f32_rn(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023;
    if (e < -126 || e > 127) return __uint_as_float(f32_rn_rare(b));
    unsigned f = ((unsigned)(e + 127) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned r = lo & 0x1fffffffu;
    f += (r > 0x10000000u || (r == 0x10000000u && (f & 1u))) ? 1u : 0u;
    return __uint_as_float((hi & 0x80000000u) | f);
}

// max of two non-negative doubles by their bit patterns (same order as the
// values for +0 and positive finite numbers), off the FP64 pipe
__device__ __forceinline__ double max_nonneg(double a, double b)
{
    return __double_as_longlong(b) > __double_as_longlong(a) ? b : a;
}

__device__ inline void write_records(const MomArgs &A, const Frame &fr, int node, int level, bool leaf, int link,
                                     int cnt, const uint32_t lo[3], const uint32_t hi[3], double M,
                                     const double com[3], const double Q[6], const double S[6], double hmax,
                                     const double c[3], const int ci[3])
{
    uint32_t cq[3];
    for (int a = 0; a < 3; a++) cq[a] = cell_of(com[a], fr.x0[a], fr.scale);
    A.W0[node] = make_int4((int)lo[0], (int)lo[1], (int)lo[2], level | (leaf ? 256 : 0));
    A.W1[node] = make_int4((int)hi[0], (int)hi[1], (int)hi[2], link);
    A.W2[node] = make_int4((int)cq[0], (int)cq[1], (int)cq[2], cnt);
    A.Whq[node] = hq_of(hmax, fr.scale);
    A.E0[node] = make_float4(f32_rn(com[0] - c[0]), f32_rn(com[1] - c[1]), f32_rn(com[2] - c[2]), f32_rn(M));
    A.E1[node] = make_float4(f32_rn(Q[0]), f32_rn(Q[1]), f32_rn(Q[3]), f32_rn(Q[4]));
    A.E2[node] = make_float4(f32_rn(Q[5]), __int_as_float(ci[0]), __int_as_float(ci[1]), __int_as_float(ci[2]));
    A.nM[node] = M;
    for (int a = 0; a < 3; a++) A.ncom[3 * (size_t)node + a] = com[a];
    for (int k = 0; k < 6; k++) A.nQ[6 * (size_t)node + k] = Q[k];
    for (int k = 0; k < 6; k++) A.nS[6 * (size_t)node + k] = S[k];
    A.nhmax[node] = hmax;
}

// Moments about the node's cell centre c, then moved to the centre of mass
// (parallel-axis theorem): M, s = sum m (x - c), S' = sum m (x - c)(x - c)^T
// in one pass; com = c + s/M, S = S' - s (s/M)^T, Q = 3 S - tr(S) I.  The
// operation order is fixed (members in sorted order, children in octant
// order; the products added into S' and the shift are explicit fused
// multiply-adds, everything else is uncontracted), so the values are
// reproducible bit for bit.
__device__ inline void moments_finish(double M, const double s[3], double S[6], const double cen[3], double com[3],
                                      double Q[6])
{
    if (M > 0.0) {
        double dl[3];
        for (int a = 0; a < 3; a++) {
            dl[a] = s[a] / M;
            com[a] = cen[a] + dl[a];
        }
        S[0] = __fma_rn(-s[0], dl[0], S[0]);
        S[1] = __fma_rn(-s[1], dl[1], S[1]);
        S[2] = __fma_rn(-s[2], dl[2], S[2]);
        S[3] = __fma_rn(-s[0], dl[1], S[3]);
        S[4] = __fma_rn(-s[0], dl[2], S[4]);
        S[5] = __fma_rn(-s[1], dl[2], S[5]);
    } else {
        for (int a = 0; a < 3; a++) com[a] = cen[a];
    }
    double tr = S[0] + S[1] + S[2];
    Q[0] = 3.0 * S[0] - tr;
    Q[1] = 3.0 * S[1] - tr;
    Q[2] = 3.0 * S[2] - tr;
    Q[3] = 3.0 * S[3];
    Q[4] = 3.0 * S[4];
    Q[5] = 3.0 * S[5];
}

// Member data of a leaf: from the chunk staged in shared memory where it
// holds them (ranks [c0, lim)), else from global memory.
struct LeafSrc {
    const MomArgs &A;
    const double *sxyz, *smass; // staged positions and masses of ranks [c0, lim), or none
    int c0, lim;
    __device__ bool in(int k) const { return k >= c0 && k < lim; }
    __device__ uint64_t key(int k) const { return __ldg(&A.key[k]); }
    __device__ double x(int k, int a) const { return in(k) ? sxyz[3 * (k - c0) + a] : A.pos[3 * (size_t)k + a]; }
    __device__ double mass(int k) const { return in(k) ? smass[k - c0] : A.mass[k]; }
    __device__ double soft(int k) const { return __ldg(&A.soft[k]); }
    __device__ bool sink(int k) const { return __ldg(&A.sink[k]) != 0; }
};

__device__ void leaf_moments(const MomArgs &A, const LeafSrc &D, const Frame &fr, int node)
{
    const int f = A.nfirst[node], c = A.ncount[node], level = A.nlevel[node];
    uint32_t lo[3] = {SFG_GRID_MAX, SFG_GRID_MAX, SFG_GRID_MAX}, hi[3] = {0, 0, 0};
    int ci[3];
    double cen[3];
    {
        // every member shares the cell prefix: the first one gives the centre
        uint64_t key = D.key(f);
        uint32_t q[3] = {compact3(key >> 2), compact3(key >> 1), compact3(key)};
        node_centre(fr, q, level, ci, cen);
    }
    double M = 0.0, s[3] = {0.0, 0.0, 0.0}, S[6] = {0, 0, 0, 0, 0, 0}, hmax = 0.0;
    for (int k = f; k < f + c; k++) {
        double m = D.mass(k);
        double d[3], md[3];
        for (int a = 0; a < 3; a++) d[a] = D.x(k, a) - cen[a];
        M = M + m;
        for (int a = 0; a < 3; a++) md[a] = m * d[a];
        for (int a = 0; a < 3; a++) s[a] = s[a] + md[a];
        S[0] = __fma_rn(md[0], d[0], S[0]);
        S[1] = __fma_rn(md[1], d[1], S[1]);
        S[2] = __fma_rn(md[2], d[2], S[2]);
        S[3] = __fma_rn(md[0], d[1], S[3]);
        S[4] = __fma_rn(md[0], d[2], S[4]);
        S[5] = __fma_rn(md[1], d[2], S[5]);
        uint64_t key = D.key(k);
        uint32_t q[3] = {compact3(key >> 2), compact3(key >> 1), compact3(key)};
        for (int a = 0; a < 3; a++) {
            lo[a] = q[a] < lo[a] ? q[a] : lo[a];
            hi[a] = q[a] > hi[a] ? q[a] : hi[a];
        }
        double h = D.soft(k);
        hmax = max_nonneg(hmax, h);
        // particle record of the walk: FP32 offset from the leaf centre
        float hs = f32_rn(h);
        if (D.sink(k)) hs = -hs;
        A.pw[k] = make_float4(f32_rn(d[0]), f32_rn(d[1]), f32_rn(d[2]), f32_rn(m));
        A.pc[k] = make_int4(ci[0], ci[1], ci[2], __float_as_int(hs));
        A.pleaf[k] = node;
    }
    double com[3], Q[6];
    moments_finish(M, s, S, cen, com, Q);
    write_records(A, fr, node, level, true, f, c, lo, hi, M, com, Q, S, hmax, cen, ci);
}

__device__ void internal_moments(const MomArgs &A, const Frame &fr, int node)
{
    const int cf = A.nchild_first[node], nc = A.nnchild[node], level = A.nlevel[node];
    uint32_t lo[3] = {SFG_GRID_MAX, SFG_GRID_MAX, SFG_GRID_MAX}, hi[3] = {0, 0, 0};
    double hmax = 0.0;
    for (int k = 0; k < nc; k++) {
        int ch = cf + k;
        int4 w0 = __ldcg(&A.W0[ch]), w1 = __ldcg(&A.W1[ch]);
        uint32_t l3[3] = {(uint32_t)w0.x, (uint32_t)w0.y, (uint32_t)w0.z};
        uint32_t h3[3] = {(uint32_t)w1.x, (uint32_t)w1.y, (uint32_t)w1.z};
        for (int a = 0; a < 3; a++) {
            lo[a] = l3[a] < lo[a] ? l3[a] : lo[a];
            hi[a] = h3[a] > hi[a] ? h3[a] : hi[a];
        }
        hmax = max_nonneg(hmax, __ldcg(&A.nhmax[ch]));
    }
    int ci[3];
    double cen[3];
    node_centre(fr, lo, level, ci, cen);
    double M = 0.0, s[3] = {0.0, 0.0, 0.0}, S[6] = {0, 0, 0, 0, 0, 0};
    for (int k = 0; k < nc; k++) {
        int ch = cf + k;
        double Mc = __ldcg(&A.nM[ch]);
        double d[3], md[3];
        for (int a = 0; a < 3; a++) d[a] = __ldcg(&A.ncom[3 * (size_t)ch + a]) - cen[a];
        M = M + Mc;
        for (int a = 0; a < 3; a++) md[a] = Mc * d[a];
        for (int a = 0; a < 3; a++) s[a] = s[a] + md[a];
        const double *Sc = A.nS + 6 * (size_t)ch;
        S[0] = S[0] + __fma_rn(md[0], d[0], __ldcg(&Sc[0]));
        S[1] = S[1] + __fma_rn(md[1], d[1], __ldcg(&Sc[1]));
        S[2] = S[2] + __fma_rn(md[2], d[2], __ldcg(&Sc[2]));
        S[3] = S[3] + __fma_rn(md[0], d[1], __ldcg(&Sc[3]));
        S[4] = S[4] + __fma_rn(md[0], d[2], __ldcg(&Sc[4]));
        S[5] = S[5] + __fma_rn(md[1], d[2], __ldcg(&Sc[5]));
    }
    double com[3], Q[6];
    moments_finish(M, s, S, cen, com, Q);
    write_records(A, fr, node, level, false, cf, nc, lo, hi, M, com, Q, S, hmax, cen, ci);
}

// Leaves: a lane sums one leaf in member order, and a warp runs as long as
// its largest leaf, so a warp's lanes take leaves of about the same size.
// Below LM_STAGED_MIN particles (the particle arrays about L2-resident) one
// launch takes every leaf from a list ordered by member count.  Above it,
// where those scattered member reads go to DRAM, blocks take chunks of
// LM_CH sorted ranks: the chunk's positions and masses (and the next LM_EXT
// ranks', where its last leaves end) are staged in shared memory with
// coalesced loads, and its leaves -- those starting in the chunk -- are taken
// largest first; keys, softenings and sink flags (17 of the 49 bytes a member
// needs) are read through the read-only cache instead, so that three blocks
// fit on an SM (the 2e7-particle build went from 6.54 to 6.36 ms against
// staging everything at two blocks per SM).  Then internal nodes one
// level at a time from the deepest (one thread per node; its children are
// final).
constexpr int LM_CH = 2048, LM_EXT = 64, LM_SPAN = LM_CH + LM_EXT, LM_BT = 256, LM_BINS = 64; // 3 blocks per SM
constexpr size_t LM_SMEM = (size_t)LM_SPAN * (3 * 8 + 8);
constexpr int64_t LM_STAGED_MIN = 1 << 22;

__global__ void k_leaf_moments(MomArgs A, const int *leaves)
{
    const LeafSrc D{A, nullptr, nullptr, 0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.nn; i += gridDim.x * blockDim.x) {
        const int node = leaves[i];
        if (node >= 0) leaf_moments(A, D, A.fr[A.ncloud[node]], node);
    }
}

// lstart[rank] = the leaf whose first member is at that rank (else -1).
__global__ void k_leaf_starts_at(const int32_t *nnchild, const int32_t *nfirst, int nn, int *lstart)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x)
        if (nnchild[i] == 0) lstart[nfirst[i]] = i;
}

__global__ void __launch_bounds__(LM_BT) k_leaf_moments_staged(MomArgs A, const int *lstart, int n)
{
    extern __shared__ __align__(16) unsigned char lm_smem[];
    double *sxyz = (double *)lm_smem;
    double *smass = sxyz + 3 * LM_SPAN;
    __shared__ int slist[LM_CH];
    __shared__ int hist[LM_BINS], nleaf;
    for (int c0 = blockIdx.x * LM_CH; c0 < n; c0 += gridDim.x * LM_CH) {
        const int lim = min(n, c0 + LM_SPAN);
        const int span = lim - c0;
        for (int q = threadIdx.x; q < 3 * span; q += LM_BT) sxyz[q] = A.pos[3 * (size_t)c0 + q];
        for (int q = threadIdx.x; q < span; q += LM_BT) smass[q] = A.mass[c0 + q];
        if (threadIdx.x < LM_BINS) hist[threadIdx.x] = 0;
        __syncthreads();
        // the chunk's leaves by member count (bin 0 = the largest)
        constexpr int PER = LM_CH / LM_BT;
        int id[PER], bin[PER];
#pragma unroll
        for (int r = 0; r < PER; r++) {
            const int k = c0 + r * LM_BT + threadIdx.x;
            id[r] = k < n ? lstart[k] : -1;
            bin[r] = 0;
            if (id[r] >= 0) {
                bin[r] = LM_BINS - min(max(A.ncount[id[r]], 1), LM_BINS);
                atomicAdd(&hist[bin[r]], 1);
            }
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            int a = hist[lane], b = hist[lane + 32], ia = a, ib = b;
            for (int o = 1; o < 32; o <<= 1) {
                const int ta = __shfl_up_sync(0xffffffffu, ia, o), tb = __shfl_up_sync(0xffffffffu, ib, o);
                if (lane >= o) {
                    ia += ta;
                    ib += tb;
                }
            }
            const int tot_a = __shfl_sync(0xffffffffu, ia, 31);
            hist[lane] = ia - a;
            hist[lane + 32] = tot_a + ib - b;
            if (lane == 31) nleaf = tot_a + ib;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < PER; r++)
            if (id[r] >= 0) slist[atomicAdd(&hist[bin[r]], 1)] = id[r];
        __syncthreads();
        const LeafSrc D{A, sxyz, smass, c0, lim};
        for (int q = threadIdx.x; q < nleaf; q += LM_BT) {
            const int node = slist[q];
            leaf_moments(A, D, A.fr[A.ncloud[node]], node);
        }
        __syncthreads();
    }
}

// Node order of the internal passes: within every level, internal nodes by
// child count (8 first), then the leaves.  A lane combines one node's
// children, so a warp's lanes take nodes of the same child count; in
// breadth-first order leaves and internal nodes interleave (clumpy clouds:
// about a quarter of the lanes busy).  A node's sums do not depend on its
// slot, and every level keeps its slice [lvl_off[l], lvl_off[l + 1]).
constexpr int NB_BINS = (SFG_LMAX + 1) * 9;

__device__ __forceinline__ int node_bin(int level, int nch) { return level * 9 + (8 - min(max(nch, 0), 8)); }

__global__ void k_node_hist(const int32_t *nlevel, const int32_t *nnchild, int nn, unsigned *hist)
{
    __shared__ unsigned h[NB_BINS];
    for (int b = threadIdx.x; b < NB_BINS; b += blockDim.x) h[b] = 0;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x)
        atomicAdd(&h[node_bin(nlevel[i], nnchild[i])], 1u);
    __syncthreads();
    for (int b = threadIdx.x; b < NB_BINS; b += blockDim.x)
        if (h[b]) atomicAdd(&hist[b], h[b]);
}

__global__ void k_node_starts(const unsigned *hist, unsigned *cur)
{
    unsigned run = 0;
    for (int b = 0; b < NB_BINS; b++) {
        cur[b] = run;
        run += hist[b];
    }
}

__global__ void k_node_scatter(const int32_t *nlevel, const int32_t *nnchild, int nn, unsigned *cur, int *perm)
{
    __shared__ unsigned h[NB_BINS], base[NB_BINS];
    for (int c0 = blockIdx.x * blockDim.x; c0 < nn; c0 += gridDim.x * blockDim.x) {
        for (int b = threadIdx.x; b < NB_BINS; b += blockDim.x) h[b] = 0;
        __syncthreads();
        const int i = c0 + threadIdx.x;
        int bin = -1;
        unsigned r = 0;
        if (i < nn) {
            bin = node_bin(nlevel[i], nnchild[i]);
            r = atomicAdd(&h[bin], 1u);
        }
        __syncthreads();
        for (int b = threadIdx.x; b < NB_BINS; b += blockDim.x)
            if (h[b]) base[b] = atomicAdd(&cur[b], h[b]);
        __syncthreads();
        if (bin >= 0) perm[base[bin] + r] = i;
        __syncthreads();
    }
}

__global__ void k_internal_moments(MomArgs A, const int *perm, int b, int e)
{
    for (int i = b + blockIdx.x * blockDim.x + threadIdx.x; i < e; i += gridDim.x * blockDim.x) {
        const int node = perm[i];
        if (A.nnchild[node] != 0) internal_moments(A, A.fr[A.ncloud[node]], node);
    }
}

// Nodes per level taken by the single-block pass.  A node's combine is ~200
// FP64 operations and one SM retires 2 per clock, so a level in one block
// costs about as much as a launch of its own at ~64 nodes.
constexpr int SMALL_LEVEL = 64;

// The small top levels (0..top) in one block, deepest first, a barrier
// between levels (the children of a level are final before it starts).
struct LevelOffsets {
    int off[SFG_LMAX + 3];
};

__global__ void __launch_bounds__(256) k_internal_moments_top(MomArgs A, const int *perm, LevelOffsets L, int top)
{
    for (int l = top; l >= 0; l--) {
        for (int i = L.off[l] + threadIdx.x; i < L.off[l + 1]; i += blockDim.x) {
            const int node = perm[i];
            if (A.nnchild[node] != 0) internal_moments(A, A.fr[A.ncloud[node]], node);
        }
        __syncthreads();
    }
}

// Leaf ids ordered by member count, largest first (the slots past the leaf
// count hold -1).  A lane sums one leaf, so a warp runs as long as its
// largest leaf: in node order the counts of neighbouring leaves differ
// widely (clumpy clouds: ~40% of the lanes busy), by count they match.
// A leaf's sums do not depend on where it sits in the list.
constexpr int LB_BINS = 64; // counts 1..63, and >= 64 together

__device__ __forceinline__ int leaf_bin(int count)
{
    return LB_BINS - min(max(count, 1), LB_BINS); // bin 0 = the largest leaves
}

__global__ void k_leaf_hist(const int32_t *nnchild, const int32_t *ncount, int nn, unsigned *hist)
{
    __shared__ unsigned h[LB_BINS];
    for (int b = threadIdx.x; b < LB_BINS; b += blockDim.x) h[b] = 0;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x)
        if (nnchild[i] == 0) atomicAdd(&h[leaf_bin(ncount[i])], 1u);
    __syncthreads();
    for (int b = threadIdx.x; b < LB_BINS; b += blockDim.x)
        if (h[b]) atomicAdd(&hist[b], h[b]);
}

// exclusive prefix of the bins (one warp)
__global__ void k_leaf_starts(const unsigned *hist, unsigned *cur)
{
    const int lane = threadIdx.x;
    unsigned a = hist[lane], b = hist[lane + 32];
    unsigned ia = a, ib = b;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned ta = __shfl_up_sync(0xffffffffu, ia, o), tb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) {
            ia += ta;
            ib += tb;
        }
    }
    const unsigned tot_a = __shfl_sync(0xffffffffu, ia, 31);
    cur[lane] = ia - a;
    cur[lane + 32] = tot_a + ib - b;
}

// one block-wide chunk of nodes per iteration: ranks within the chunk from
// shared counters, the chunk's range of each bin from one global atomic
__global__ void k_leaf_scatter(const int32_t *nnchild, const int32_t *ncount, int nn, unsigned *cur, int *leaves)
{
    __shared__ unsigned h[LB_BINS], base[LB_BINS];
    for (int c0 = blockIdx.x * blockDim.x; c0 < nn; c0 += gridDim.x * blockDim.x) {
        for (int b = threadIdx.x; b < LB_BINS; b += blockDim.x) h[b] = 0;
        __syncthreads();
        const int i = c0 + threadIdx.x;
        int bin = -1;
        unsigned r = 0;
        if (i < nn && nnchild[i] == 0) {
            bin = leaf_bin(ncount[i]);
            r = atomicAdd(&h[bin], 1u);
        }
        __syncthreads();
        for (int b = threadIdx.x; b < LB_BINS; b += blockDim.x)
            if (h[b]) base[b] = atomicAdd(&cur[b], h[b]);
        __syncthreads();
        if (bin >= 0) leaves[base[bin] + r] = i;
        __syncthreads();
    }
}

// ------------------------------------------------------------ host side ----
static int grid_for(int64_t n, int bt)
{
    int64_t g = (n + bt - 1) / bt;
    int64_t cap = (int64_t)num_sms() * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

#define ALLOC(ptr, type, count)                                                                              \
    do {                                                                                                     \
        ptr = (type *)dev_alloc(t, sizeof(type) * (size_t)(count), s);                                      \
        if (!ptr) return SFG_ENOMEM;                                                                         \
    } while (0)

static int alloc_nodes(Tree *t, int cap, cudaStream_t s)
{
    t->cap = cap;
    ALLOC(t->nfirst, int32_t, cap);
    ALLOC(t->ncount, int32_t, cap);
    ALLOC(t->nparent, int32_t, cap);
    ALLOC(t->nchild_first, int32_t, cap);
    ALLOC(t->nnchild, int32_t, cap);
    ALLOC(t->nlevel, int32_t, cap);
    ALLOC(t->ncloud, int32_t, cap);
    return SFG_OK;
}

static void free_nodes(Tree *t, cudaStream_t s)
{
    dev_free(t, t->nfirst, s);
    dev_free(t, t->ncount, s);
    dev_free(t, t->nparent, s);
    dev_free(t, t->nchild_first, s);
    dev_free(t, t->nnchild, s);
    dev_free(t, t->nlevel, s);
    dev_free(t, t->ncloud, s);
    t->nfirst = t->ncount = t->nparent = t->nchild_first = t->nnchild = t->nlevel = t->ncloud = nullptr;
}

// Launch grid (chunks, C) whose blocks each stride over one cloud's range.
static dim3 cloud_grid(const Tree *t, int bt)
{
    int64_t big = 1;
    for (int c = 0; c < t->nclouds; c++) big = std::max(big, t->off_h[c + 1] - t->off_h[c]);
    int64_t chunks = (big + bt - 1) / bt;
    int64_t cap = std::max<int64_t>(1, (int64_t)num_sms() * 8 / t->nclouds);
    return dim3((unsigned)std::max<int64_t>(1, std::min(chunks, cap)), (unsigned)t->nclouds);
}

int build_tree(Tree *t, const double *pos, const double *mass, const double *soft, const uint8_t *is_sink,
               cudaStream_t s)
{
    const int n = (int)t->n;
    const int C = t->nclouds;
    const int BT = 256;
    ALLOC(t->d_status, int, 1);
    ALLOC(t->d_frame, Frame, C);
    ALLOC(t->d_off, int64_t, C + 1);
    ALLOC(t->d_minmax, unsigned long long, 6 * (size_t)C);
    ALLOC(t->d_lvl, int, SFG_LMAX + 3);
    ALLOC(t->d_counters, unsigned long long, NCOUNTERS);
    ALLOC(t->d_n, int, 1);
    SFG_CUDA_OK(cudaMemcpyAsync(t->d_off, t->off_h.data(), sizeof(int64_t) * (C + 1), cudaMemcpyHostToDevice, s));
    k_set_int<<<1, 1, 0, s>>>(t->d_n, n);
    SFG_CUDA_OK(cudaMemsetAsync(t->d_status, 0, sizeof(int), s));
    SFG_CUDA_OK(cudaMemsetAsync(t->d_counters, 0, NCOUNTERS * sizeof(unsigned long long), s));

    const dim3 cg = cloud_grid(t, BT);
    t->n_launch += 2 + 3; // k_set_int, k_minmax_init, k_validate_minmax, k_frame, k_keys
    k_minmax_init<<<grid_for(6 * C, BT), BT, 0, s>>>(t->d_minmax, C);
    k_validate_minmax<<<cg, BT, 0, s>>>(pos, mass, soft, t->d_off, t->d_minmax, t->d_status);
    k_frame<<<(C + 127) / 128, 128, 0, s>>>(t->d_minmax, t->d_frame, C, t->d_status);

    // keys + sort: 8 passes on the Morton key, then (several clouds) stable
    // passes on the cloud id, so each cloud is contiguous and key-sorted
    uint64_t *k0, *k1;
    uint32_t *v0, *v1;
    uint16_t *cloud_of = nullptr;
    ALLOC(k0, uint64_t, n);
    ALLOC(k1, uint64_t, n);
    ALLOC(v0, uint32_t, n);
    ALLOC(v1, uint32_t, n);
    if (C > 1) ALLOC(cloud_of, uint16_t, n);
    k_keys<<<cg, BT, 0, s>>>(pos, t->d_off, t->d_frame, k0, v0, cloud_of);
    const int nb = (n + OS_TILE - 1) / OS_TILE;
    unsigned *gcount, *gstart, *tile_ctr;
    unsigned long long *look;
    ALLOC(gcount, unsigned, RS_MAXPASS * 256);
    ALLOC(gstart, unsigned, RS_MAXPASS * 256);
    ALLOC(tile_ctr, unsigned, RS_MAXPASS);
    ALLOC(look, unsigned long long, 256 * (size_t)nb);
    const int cloud_passes = C <= 1 ? 0 : (C <= 256 ? 1 : 2);
    const int npass = 8 + cloud_passes;
    SFG_CUDA_OK(cudaMemsetAsync(gcount, 0, sizeof(unsigned) * RS_MAXPASS * 256, s));
    SFG_CUDA_OK(cudaMemsetAsync(tile_ctr, 0, sizeof(unsigned) * RS_MAXPASS, s));
    k_rs_count_all<<<std::min(nb, num_sms() * 2), 256, 0, s>>>(k0, n, cloud_of, cloud_passes, gcount);
    k_rs_start<<<1, 256, 0, s>>>(gcount, npass, gstart);
    t->n_launch += 2 + npass + 1; // counts, starts, one launch per pass, pack
    for (int pass = 0; pass < npass; pass++) {
        const bool by_cloud = pass >= 8;
        int shift = by_cloud ? 8 * (pass - 8) : 8 * pass;
        const uint16_t *cl = by_cloud ? cloud_of : nullptr;
        SFG_CUDA_OK(cudaMemsetAsync(look, 0, sizeof(unsigned long long) * 256 * (size_t)nb, s));
        k_rs_onesweep<<<nb, RS_WARPS * 32, 0, s>>>(k0, v0, k1, v1, n, shift, cl, gstart + 256 * pass, look,
                                                   tile_ctr + pass, t->d_status);
        uint64_t *tk = k0;
        k0 = k1;
        k1 = tk;
        uint32_t *tv = v0;
        v0 = v1;
        v1 = tv;
    }
    t->key = k0;
    dev_free(t, k1, s);
    dev_free(t, gcount, s);
    dev_free(t, gstart, s);
    dev_free(t, tile_ctr, s);
    dev_free(t, look, s);

    ALLOC(t->order, int32_t, n);
    ALLOC(t->rank, int32_t, n);
    ALLOC(t->pos_s, double, 3 * (size_t)n);
    ALLOC(t->mass_s, double, n);
    ALLOC(t->soft_s, double, n);
    ALLOC(t->sink_s, uint8_t, n);
    ALLOC(t->pw, float4, n);
    ALLOC(t->pc, int4, n);
    ALLOC(t->pleaf, int32_t, n);
    if (C > 1) ALLOC(t->pcloud, int32_t, n);
    k_pack<<<grid_for(n, BT), BT, 0, s>>>(pos, mass, soft, is_sink, n, v0, t->order, t->rank, t->pos_s, t->mass_s,
                                          t->soft_s, t->sink_s, cloud_of, t->pcloud);
    dev_free(t, v0, s);
    dev_free(t, v1, s);
    dev_free(t, cloud_of, s);

    // octree, retried with a larger node capacity if the estimate was short
    // measured on uniform and clumpy clouds: nodes / n <= 1.5, 0.77, 0.52,
    // 0.32, 0.16 for leaf sizes 1, 4, 8, 16, 32
    int64_t cap64 = 6 * ((int64_t)n / (t->prm.leaf_size + 2)) + 4096 + 64 * (int64_t)C;
    int *tmp = nullptr, *tmpo = nullptr, *bnd = nullptr;
    uint64_t *ks = nullptr;
    ALLOC(ks, uint64_t, (n + KS - 1) / KS);
    k_key_samples<<<grid_for((n + KS - 1) / KS, BT), BT, 0, s>>>(t->key, n, ks);
    t->n_launch += 1;
    for (int attempt = 0;; attempt++) {
        if (cap64 > 0x7fffffff) cap64 = 0x7fffffff;
        int cap = (int)cap64;
        int rc = alloc_nodes(t, cap, s);
        if (rc) return rc;
        ALLOC(tmp, int, cap + 1);
        ALLOC(tmpo, int, cap + 1);
        ALLOC(bnd, int, 7 * (size_t)cap);
        char *scr = nullptr;
        ALLOC(scr, char, scan1p_bytes(cap));
        Scan1P sc;
        sc.init(scr, cap, s);
        k_oct_root<<<(C + 127) / 128, 128, 0, s>>>(t->d_off, C, t->nfirst, t->ncount, t->nparent, t->nlevel,
                                                   t->ncloud, t->d_lvl);
        t->n_launch += 1 + (SFG_LMAX + 1) * 3; // roots; per level: count, scan, write
        // grid-stride over a level (its size is only known on the device)
        const int og = std::min(grid_for(cap, BT), num_sms() * 4);
        auto levels = [&](int l0, int l1) {
            for (int level = l0; level < l1; level++) {
                k_oct_count<<<og, BT, 0, s>>>(t->key, ks, t->d_lvl, level, t->prm.leaf_size, cap, t->nfirst,
                                              t->ncount, tmp, bnd, t->d_status);
                sc.range(tmp, tmpo, t->d_lvl + level, t->d_lvl + level + 1, cap, t->d_lvl + level + 2,
                         t->d_lvl + level + 1, t->d_status, s);
                k_oct_write<<<og, BT, 0, s>>>(bnd, t->d_lvl, level, t->prm.leaf_size, cap, t->nfirst, t->ncount,
                                              t->nparent, t->nchild_first, t->nnchild, t->nlevel, t->ncloud, tmpo,
                                              t->d_status);
            }
        };
        // the levels the last tree needed (and two more) first; then the rest
        // only if the tree goes deeper (their launches find empty levels)
        const int l1 = std::min(SFG_LMAX + 1, g_depth_hint.load() + 2);
        levels(0, l1);
        int st = 0;
        SFG_CUDA_OK(cudaMemcpyAsync(&st, t->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
        SFG_CUDA_OK(cudaMemcpyAsync(t->lvl_off, t->d_lvl, sizeof(int) * (SFG_LMAX + 3), cudaMemcpyDeviceToHost, s));
        SFG_CUDA_OK(cudaStreamSynchronize(s));
        SFG_CUDA_OK(cudaGetLastError());
        if (l1 <= SFG_LMAX && !(st & (ST_NODECAP | ST_EINVAL))) {
            if (t->lvl_off[l1 + 1] > t->lvl_off[l1]) {
                levels(l1, SFG_LMAX + 1);
                SFG_CUDA_OK(cudaMemcpyAsync(&st, t->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
                SFG_CUDA_OK(
                    cudaMemcpyAsync(t->lvl_off, t->d_lvl, sizeof(int) * (SFG_LMAX + 3), cudaMemcpyDeviceToHost, s));
                SFG_CUDA_OK(cudaStreamSynchronize(s));
                SFG_CUDA_OK(cudaGetLastError());
            } else {
                // level l1 is empty, and so is every deeper one
                t->n_launch -= (SFG_LMAX + 1 - l1) * 3;
                for (int l = l1 + 2; l <= SFG_LMAX + 2; l++) t->lvl_off[l] = t->lvl_off[l1 + 1];
            }
        }
        dev_free(t, tmp, s);
        dev_free(t, tmpo, s);
        dev_free(t, bnd, s);
        dev_free(t, scr, s);
        if (st & ST_EINVAL) return SFG_EINVAL;
        if (!(st & ST_NODECAP)) break;
        free_nodes(t, s);
        SFG_CUDA_OK(cudaMemsetAsync(t->d_status, 0, sizeof(int), s));
        cap64 *= 2;
        if (attempt > 8) return SFG_ENOMEM;
    }
    dev_free(t, ks, s);
    const int nn = t->lvl_off[SFG_LMAX + 2];
    t->nn = nn;
    t->depth = 0;
    for (int l = 0; l <= SFG_LMAX; l++)
        if (t->lvl_off[l + 1] > t->lvl_off[l]) t->depth = l;
    t->n_levels = t->depth + 1;
    g_depth_hint.store(t->depth);

    ALLOC(t->W0, int4, nn);
    ALLOC(t->W1, int4, nn);
    ALLOC(t->W2, int4, nn);
    ALLOC(t->Whq, unsigned long long, nn);
    ALLOC(t->E0, float4, nn);
    ALLOC(t->E1, float4, nn);
    ALLOC(t->E2, float4, nn);
    ALLOC(t->nM, double, nn);
    ALLOC(t->ncom, double, 3 * (size_t)nn);
    ALLOC(t->nQ, double, 6 * (size_t)nn);
    ALLOC(t->nhmax, double, nn);
    const bool staged = n >= LM_STAGED_MIN;
    int *lidx = nullptr; // staged: leaf starting at each rank; else the leaves by member count
    unsigned *lhist = nullptr;
    double *nS;
    ALLOC(nS, double, 6 * (size_t)nn);
    if (staged) {
        ALLOC(lidx, int, n);
        SFG_CUDA_OK(cudaMemsetAsync(lidx, 0xff, sizeof(int) * (size_t)n, s));
        k_leaf_starts_at<<<grid_for(nn, BT), BT, 0, s>>>(t->nnchild, t->nfirst, nn, lidx);
        t->n_launch += 1;
    } else {
        ALLOC(lidx, int, nn);
        ALLOC(lhist, unsigned, 2 * LB_BINS);
        SFG_CUDA_OK(cudaMemsetAsync(lidx, 0xff, sizeof(int) * (size_t)nn, s));
        SFG_CUDA_OK(cudaMemsetAsync(lhist, 0, sizeof(unsigned) * LB_BINS, s));
        k_leaf_hist<<<grid_for(nn, BT), BT, 0, s>>>(t->nnchild, t->ncount, nn, lhist);
        k_leaf_starts<<<1, 32, 0, s>>>(lhist, lhist + LB_BINS);
        k_leaf_scatter<<<grid_for(nn, BT), BT, 0, s>>>(t->nnchild, t->ncount, nn, lhist + LB_BINS, lidx);
        t->n_launch += 3;
    }
    MomArgs A;
    A.key = t->key;
    A.pos = t->pos_s;
    A.mass = t->mass_s;
    A.soft = t->soft_s;
    A.sink = t->sink_s;
    A.nfirst = t->nfirst;
    A.ncount = t->ncount;
    A.nparent = t->nparent;
    A.nchild_first = t->nchild_first;
    A.nnchild = t->nnchild;
    A.nlevel = t->nlevel;
    A.ncloud = t->ncloud;
    A.fr = t->d_frame;
    A.W0 = t->W0;
    A.W1 = t->W1;
    A.W2 = t->W2;
    A.Whq = t->Whq;
    A.E0 = t->E0;
    A.E1 = t->E1;
    A.E2 = t->E2;
    A.nM = t->nM;
    A.ncom = t->ncom;
    A.nQ = t->nQ;
    A.nhmax = t->nhmax;
    A.nS = nS;
    A.pw = t->pw;
    A.pc = t->pc;
    A.pleaf = t->pleaf;
    A.nn = nn;
    if (staged) {
        // the staged chunk needs more than the default 48 KB of shared memory
        SFG_CUDA_OK(cudaFuncSetAttribute(k_leaf_moments_staged, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LM_SMEM));
        const int chunks = (int)((n + LM_CH - 1) / LM_CH);
        k_leaf_moments_staged<<<std::min(chunks, 3 * num_sms()), LM_BT, LM_SMEM, s>>>(A, lidx, (int)n);
    } else {
        k_leaf_moments<<<grid_for(nn, 128), 128, 0, s>>>(A, lidx);
    }
    t->n_launch += 1;
    int *perm = nullptr;
    unsigned *nbin = nullptr;
    ALLOC(perm, int, nn);
    ALLOC(nbin, unsigned, 2 * NB_BINS);
    SFG_CUDA_OK(cudaMemsetAsync(nbin, 0, sizeof(unsigned) * NB_BINS, s));
    k_node_hist<<<grid_for(nn, BT), BT, 0, s>>>(t->nlevel, t->nnchild, nn, nbin);
    k_node_starts<<<1, 1, 0, s>>>(nbin, nbin + NB_BINS);
    k_node_scatter<<<grid_for(nn, BT), BT, 0, s>>>(t->nlevel, t->nnchild, nn, nbin + NB_BINS, perm);
    t->n_launch += 3;
    // levels 0..top hold few nodes each: one block takes them in one launch
    int top = -1;
    while (top + 1 < t->depth && t->lvl_off[top + 2] - t->lvl_off[top + 1] <= SMALL_LEVEL) top++;
    for (int l = t->depth - 1; l > top; l--) {
        int b = t->lvl_off[l], e = t->lvl_off[l + 1];
        // one warp per block on the smaller levels, so that they spread over the SMs
        const int bs = e - b <= num_sms() * 128 ? 32 : 128;
        k_internal_moments<<<(e - b + bs - 1) / bs, bs, 0, s>>>(A, perm, b, e);
        t->n_launch += 1;
    }
    if (top >= 0) {
        LevelOffsets L;
        for (int l = 0; l < SFG_LMAX + 3; l++) L.off[l] = t->lvl_off[l];
        k_internal_moments_top<<<1, SMALL_LEVEL, 0, s>>>(A, perm, L, top);
        t->n_launch += 1;
    }
    dev_free(t, nS, s);
    dev_free(t, perm, s);
    dev_free(t, nbin, s);
    dev_free(t, lidx, s);
    if (lhist) dev_free(t, lhist, s);
    t->frames_h.resize(C);
    SFG_CUDA_OK(cudaMemcpyAsync(t->frames_h.data(), t->d_frame, sizeof(Frame) * C, cudaMemcpyDeviceToHost, s));
    SFG_CUDA_OK(cudaStreamSynchronize(s));
    t->frame_h = t->frames_h[0];
    SFG_CUDA_OK(cudaGetLastError());
    return SFG_OK;
}

} // namespace sfg

// ------------------------------------------------ fixed-scratch key sort ----
// Frame, Morton keys and their stable sort order for up to SFG_STATIC_MAX_N
// particles, with every temporary buffer carved from one file-scope device
// array, so the call performs no device allocation.  The caller's outputs
// double as one side of the radix sort's ping-pong buffers.
namespace sfg {

constexpr int ST_NB = (SFG_STATIC_MAX_N + RS_TILE - 1) / RS_TILE;
constexpr size_t st_al(size_t x) { return (x + 255) & ~(size_t)255; } // every region starts on 256 bytes
constexpr size_t ST_OFF_MINMAX = 0;                                             // 6 x u64
constexpr size_t ST_OFF_FRAME = 256;                                            // Frame
constexpr size_t ST_OFF_HN = 512;                                               // 2 ints
constexpr size_t ST_OFF_RANGE = 768;                                            // 2 x int64: {0, n}
constexpr size_t ST_OFF_SCAN = 1024;                                            // SCAN_NB ints
constexpr size_t ST_OFF_HIST = st_al(ST_OFF_SCAN + SCAN_NB * 4);                // 256 * ST_NB ints
constexpr size_t ST_OFF_HOFF = st_al(ST_OFF_HIST + 256 * (size_t)ST_NB * 4);    // 256 * ST_NB + 1 ints
constexpr size_t ST_OFF_KEYS = st_al(ST_OFF_HOFF + (256 * (size_t)ST_NB + 1) * 4);
constexpr size_t ST_OFF_VALS = st_al(ST_OFF_KEYS + (size_t)SFG_STATIC_MAX_N * 8);
constexpr size_t ST_BYTES = st_al(ST_OFF_VALS + (size_t)SFG_STATIC_MAX_N * 4);
static_assert(ST_OFF_KEYS % 256 == 0 && ST_OFF_VALS % 256 == 0 && ST_OFF_HIST % 256 == 0, "scratch alignment");
static_assert(sizeof(Frame) <= 256 && SCAN_NB * 4 <= 4096, "scratch layout");
static_assert(ST_BYTES == 6556928, "the array size stated in sfg.h");

static __device__ __align__(256) unsigned char g_sort_scratch[ST_BYTES];

__global__ void k_minmax_pos(const double *pos, int n, unsigned long long *mm)
{
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0, 0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int a = 0; a < 3; a++) {
            unsigned long long u = ord_of(pos[3 * (size_t)i + a]);
            lo[a] = u < lo[a] ? u : lo[a];
            hi[a] = u > hi[a] ? u : hi[a];
        }
    for (int a = 0; a < 3; a++) {
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo[a], o);
            unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hi[a], o);
            lo[a] = l2 < lo[a] ? l2 : lo[a];
            hi[a] = h2 > hi[a] ? h2 : hi[a];
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&mm[a], lo[a]);
            atomicMax(&mm[3 + a], hi[a]);
        }
    }
}

__global__ void k_set_range(int64_t *range, int64_t n)
{
    range[0] = 0;
    range[1] = n;
}

// Device address of the scratch array on the current device, looked up once
// per device (the symbol's host-side name is not a device address).
static int static_scratch(unsigned char **out)
{
    static std::mutex mu;
    static unsigned char *addr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SFG_ECUDA;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SFG_ECUDA;
        }
        addr[dev] = (unsigned char *)p;
    }
    *out = addr[dev];
    return SFG_OK;
}

} // namespace sfg

extern "C" int sfg_sort_keys_static(const double *pos, int64_t n, uint64_t *key_out, int32_t *order_out,
                                    void *stream)
{
    using namespace sfg;
    if (!pos || !key_out || !order_out || n <= 0) return SFG_EINVAL;
    if (n > SFG_STATIC_MAX_N) return SFG_EINVAL;
    cudaGetLastError(); // a launch error reported at the end is this call's own
    unsigned char *base = nullptr;
    int rc = static_scratch(&base);
    if (rc != SFG_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int nn = (int)n, BT = 256;
    unsigned long long *mm = (unsigned long long *)(base + ST_OFF_MINMAX);
    Frame *fr = (Frame *)(base + ST_OFF_FRAME);
    int *hn = (int *)(base + ST_OFF_HN);
    int *scr = (int *)(base + ST_OFF_SCAN);
    int *hist = (int *)(base + ST_OFF_HIST);
    int *hoff = (int *)(base + ST_OFF_HOFF);
    uint64_t *kb = (uint64_t *)(base + ST_OFF_KEYS);
    uint32_t *vb = (uint32_t *)(base + ST_OFF_VALS);
    const int nb = (nn + RS_TILE - 1) / RS_TILE;
    // k_frame flags an unsupported extent (subnormal or beyond 2^1023) here;
    // the call does not read it back, so such inputs give unspecified keys
    int *scratch_status = hn + 1;
    int64_t *range = (int64_t *)(base + ST_OFF_RANGE);
    k_set_range<<<1, 1, 0, s>>>(range, n);
    k_set_int<<<1, 1, 0, s>>>(scratch_status, 0);
    k_minmax_init<<<1, 32, 0, s>>>(mm, 1);
    k_minmax_pos<<<grid_for(nn, BT), BT, 0, s>>>(pos, nn, mm);
    k_frame<<<1, 1, 0, s>>>(mm, fr, 1, scratch_status);
    uint64_t *ka = key_out, *kx = kb;
    uint32_t *va = (uint32_t *)order_out, *vx = vb;
    k_keys<<<dim3(grid_for(nn, BT), 1), BT, 0, s>>>(pos, range, fr, ka, va, nullptr);
    k_set_int<<<1, 1, 0, s>>>(hn, 256 * nb);
    for (int pass = 0; pass < 8; pass++) {
        int shift = 8 * pass;
        k_rs_hist<<<nb, RS_WARPS * 32, 0, s>>>(ka, va, nn, shift, hist, nb, nullptr);
        scan_exclusive(hist, hoff, hn, 256 * nb, nullptr, nullptr, scr, s);
        k_rs_scatter<<<nb, RS_WARPS * 32, 0, s>>>(ka, va, kx, vx, nn, shift, hoff, nb, nullptr);
        uint64_t *tk = ka;
        ka = kx;
        kx = tk;
        uint32_t *tv = va;
        va = vx;
        vx = tv;
    }
    // 8 passes: the sorted keys and order are back in the caller's buffers
    if (cudaGetLastError() != cudaSuccess) return SFG_ECUDA;
    return SFG_OK;
}
