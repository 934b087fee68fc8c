// api.cu -- the extern "C" entry points declared in include/sfg.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "sfg_internal.cuh"

struct sfg_tree {
    sfg::Tree t;
};

namespace sfg {

thread_local cudaError_t g_last_cuda_error = cudaSuccess;

void *dev_alloc(Tree *t, size_t bytes, cudaStream_t s)
{
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (t->prm.alloc) {
        p = t->prm.alloc(bytes, (void *)s, t->prm.alloc_ctx);
    } else if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) t->live.insert(p);
    return p;
}

void dev_free(Tree *t, void *p, cudaStream_t s)
{
    if (!p) return;
    t->live.erase(p);
    if (t->prm.alloc) {
        if (t->prm.free) t->prm.free(p, (void *)s, t->prm.alloc_ctx);
    } else {
        cudaFreeAsync(p, s);
    }
}

} // namespace sfg

using namespace sfg;

// Keep memory freed to the device's default pool mapped for reuse by later
// calls (the default release threshold returns it at every synchronization).
static void keep_pool_memory()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    static bool done[64] = {false};
    if (dev < 0 || dev >= 64 || done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done[dev] = true;
}

static void release(sfg_tree *T)
{
    Tree *t = &T->t;
    cudaStreamSynchronize(t->stream);
    for (int k = 0; k < 10; k++)
        if (t->ev[k]) cudaEventDestroy(t->ev[k]);
    std::vector<void *> ptrs(t->live.begin(), t->live.end());
    for (void *p : ptrs) dev_free(t, p, t->stream);
    cudaStreamSynchronize(t->stream);
    delete T;
}

// Modified Hermite step of sink particles (Sec. 2.3): prediction from the
// start of the step, and the correction from both evaluations (velocity
// first; the position uses the corrected velocity).  Elementwise over the
// 3 n components.
__global__ void k_hermite_predict(int64_t n3, double dt, const double *x0, const double *v0, const double *a0,
                                  const double *j0, double *xp, double *vp)
{
    const double h2 = dt * dt / 2.0, h3 = dt * dt * dt / 6.0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n3; q += (int64_t)gridDim.x * blockDim.x) {
        xp[q] = x0[q] + dt * v0[q] + h2 * a0[q] + h3 * j0[q];
        vp[q] = v0[q] + dt * a0[q] + h2 * j0[q];
    }
}

__global__ void k_hermite_correct(int64_t n3, double dt, const double *x0, const double *v0, const double *a0,
                                  const double *j0, const double *a1, const double *j1, double *x1, double *v1)
{
    const double h1 = dt / 2.0, h12 = dt * dt / 12.0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n3; q += (int64_t)gridDim.x * blockDim.x) {
        const double v = v0[q] + h1 * (a1[q] + a0[q]) + h12 * (j0[q] - j1[q]);
        x1[q] = x0[q] + h1 * (v + v0[q]) + h12 * (a0[q] - a1[q]);
        v1[q] = v;
    }
}

// Field and jerk of every particle of a sinks-only tree at (x, v).
static int sink_pass(const double *x, const double *v, const double *mass, const double *soft, const uint8_t *ones,
                     int64_t n, const sfg_params *p, cudaStream_t s, double *acc, double *jerk)
{
    sfg_tree *T = nullptr;
    int rc = sfg_build(x, mass, soft, ones, n, p, (void *)s, &T);
    if (rc != SFG_OK) return rc;
    rc = sfg_accel_jerk(T, v, nullptr, n, acc, nullptr, jerk, (void *)s);
    const int st = rc == SFG_OK ? sfg_get_status(T) : rc;
    sfg_free(T);
    return st;
}

extern "C" {

void sfg_default_params(sfg_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->G = 1.0;
    p->theta = 0.5;
    p->leaf_size = 16;
    p->group_size = 32;
    p->list_depth = 0;
    p->quadrupole = 1;
    p->precision = 0;
    p->store_lists = 1;
}

const char *sfg_last_cuda_error(void) { return cudaGetErrorName(g_last_cuda_error); }

// FMA-only probe: 8 independent chains per thread cover the FMA latency, so
// the launch runs at the FP32 pipes' issue rate; the sums are stored so that
// none of the chains is dropped.
constexpr int PK_UNROLL = 16, PK_CHAINS = 8, PK_BT = 256;

__global__ void __launch_bounds__(PK_BT) k_ffma_peak(const float *ab, int iters, float *out)
{
    const float a = ab[0], b = ab[1];
    float x[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; c++) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < PK_UNROLL; u++) {
#pragma unroll
            for (int c = 0; c < PK_CHAINS; c++) x[c] = fmaf(x[c], a, b);
        }
    }
    float sum = 0.f;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; c++) sum += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

int sfg_fp32_peak(double *tflops, double *ms, void *stream)
{
    if (!tflops) return SFG_EINVAL;
    cudaGetLastError();
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    SFG_CUDA_OK(cudaGetDevice(&dev));
    SFG_CUDA_OK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = 4 * (sms > 0 ? sms : 1), iters = 8192;
    float *buf = nullptr;
    if (cudaMallocAsync((void **)&buf, sizeof(float) * (2 + (size_t)blocks * PK_BT), s) != cudaSuccess) {
        cudaGetLastError();
        return SFG_ENOMEM;
    }
    const float ab[2] = {0.9999999f, 1e-7f};
    int rc = SFG_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float t = 0.f;
    if (cudaMemcpyAsync(buf, ab, sizeof(ab), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError());
    } else {
        k_ffma_peak<<<blocks, PK_BT, 0, s>>>(buf, iters / 4, buf + 2); // warm-up
        cudaEventRecord(e0, s);
        k_ffma_peak<<<blocks, PK_BT, 0, s>>>(buf, iters, buf + 2);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess || t <= 0.f)
            rc = cuda_fail(cudaGetLastError());
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(buf, s);
    if (rc) return rc;
    const double flops = 2.0 * (double)blocks * PK_BT * (double)iters * PK_UNROLL * PK_CHAINS;
    *tflops = flops / ((double)t * 1e-3) / 1e12;
    if (ms) *ms = (double)t;
    return SFG_OK;
}

const char *sfg_status_string(int st)
{
    switch (st) {
    case SFG_OK: return "SFG_OK";
    case SFG_EINVAL: return "SFG_EINVAL: invalid argument or input value";
    case SFG_ENOMEM: return "SFG_ENOMEM: device allocation failed";
    case SFG_ECUDA: return "SFG_ECUDA: CUDA runtime error";
    case SFG_EOVERFLOW: return "SFG_EOVERFLOW: traversal buffer overflow after retry";
    case SFG_ETIMEOUT: return "SFG_ETIMEOUT: bounded device wait expired";
    default: return "unknown sfg status";
    }
}

static int build_forest(const double *pos, const double *mass, const double *soft, const uint8_t *is_sink,
                        const int64_t *offsets, int n_clouds, const sfg_params *params, void *stream,
                        sfg_tree **out)
{
    if (!out) return SFG_EINVAL;
    *out = nullptr;
    if (!pos || !mass || !soft || !offsets || n_clouds < 1 || n_clouds > 65535) return SFG_EINVAL;
    if (offsets[0] != 0) return SFG_EINVAL;
    for (int c = 0; c < n_clouds; c++)
        if (offsets[c + 1] <= offsets[c]) return SFG_EINVAL; // every cloud holds at least one particle
    const int64_t n = offsets[n_clouds];
    if (n <= 0 || n >= 0x7fffffffLL) return SFG_EINVAL;
    sfg_params p;
    if (params) p = *params;
    else sfg_default_params(&p);
    if (!(isfinite(p.G)) || !(p.theta >= 0.0) || !isfinite(p.theta) || p.leaf_size < 1 || p.leaf_size > 256 ||
        p.group_size < 1 || p.group_size > 32 || (p.quadrupole != 0 && p.quadrupole != 1) ||
        (p.list_depth != 0 && p.list_depth != 1 && p.list_depth != 2 && p.list_depth != 4) ||
        (p.precision != 0 && p.precision != 1) || (p.alloc && !p.free))
        return SFG_EINVAL;
    cudaGetLastError();
    keep_pool_memory();
    sfg_tree *T = new sfg_tree;
    T->t.prm = p;
    T->t.n = n;
    T->t.nclouds = n_clouds;
    T->t.off_h.assign(offsets, offsets + n_clouds + 1);
    T->t.stream = (cudaStream_t)stream;
    const char *env = getenv("SFG_TIMING");
    T->t.timing = env && env[0] == '1';
    ph_begin(&T->t, PH_BUILD, (cudaStream_t)stream);
    int rc = build_tree(&T->t, pos, mass, soft, is_sink, (cudaStream_t)stream);
    ph_end(&T->t, PH_BUILD, (cudaStream_t)stream);
    if (rc != SFG_OK) {
        cudaGetLastError();
        release(T);
        return rc;
    }
    T->t.last.n = n;
    *out = T;
    return SFG_OK;
}

int sfg_build(const double *pos, const double *mass, const double *soft, const uint8_t *is_sink, int64_t n,
              const sfg_params *params, void *stream, sfg_tree **out)
{
    if (out) *out = nullptr;
    if (n <= 0 || n >= 0x7fffffffLL) return SFG_EINVAL;
    const int64_t off[2] = {0, n};
    return build_forest(pos, mass, soft, is_sink, off, 1, params, stream, out);
}

int sfg_build_batch(const double *pos, const double *mass, const double *soft, const uint8_t *is_sink,
                    const int64_t *offsets, int n_clouds, const sfg_params *params, void *stream, sfg_tree **out)
{
    return build_forest(pos, mass, soft, is_sink, offsets, n_clouds, params, stream, out);
}

int sfg_accel_batch(sfg_tree *tree, const int64_t *active_idx, int64_t n_active, double *accel, double *phi,
                    void *stream)
{
    return sfg_accel(tree, active_idx, n_active, accel, phi, stream);
}

int sfg_accel_vjp_batch(sfg_tree *tree, const int64_t *active_idx, int64_t n_active, const double *cot_a,
                        const double *cot_phi, double *d_pos, double *d_mass, void *stream)
{
    return sfg_accel_vjp(tree, active_idx, n_active, cot_a, cot_phi, d_pos, d_mass, stream);
}

int sfg_accel(sfg_tree *tree, const int64_t *active_idx, int64_t n_active, double *accel, double *phi, void *stream)
{
    if (!tree || n_active < 0 || (n_active > 0 && !accel)) return SFG_EINVAL;
    tree->t.stream = (cudaStream_t)stream;
    cudaGetLastError();
    return sfg::accel(&tree->t, active_idx, n_active, accel, phi, (cudaStream_t)stream);
}

int sfg_accel_tidal(sfg_tree *tree, const int64_t *active_idx, int64_t n_active, double *accel, double *phi,
                    double *tidal, void *stream)
{
    if (!tree || n_active < 0 || (n_active > 0 && (!accel || !tidal))) return SFG_EINVAL;
    tree->t.stream = (cudaStream_t)stream;
    cudaGetLastError();
    return sfg::accel_tidal(&tree->t, active_idx, n_active, accel, phi, tidal, (cudaStream_t)stream);
}

int sfg_accel_jerk(sfg_tree *tree, const double *vel, const int64_t *active_idx, int64_t n_active, double *accel,
                   double *phi, double *jerk, void *stream)
{
    if (!tree || !vel || n_active < 0 || (n_active > 0 && (!accel || !jerk))) return SFG_EINVAL;
    tree->t.stream = (cudaStream_t)stream;
    cudaGetLastError();
    return sfg::accel_jerk(&tree->t, vel, active_idx, n_active, accel, phi, jerk, (cudaStream_t)stream);
}

int sfg_sink_timestep(sfg_tree *tree, const double *vel, const int64_t *active_idx, int64_t n_active, double eta,
                      double *dt, void *stream)
{
    if (!tree || !vel || n_active < 0 || (n_active > 0 && !dt) || !(eta > 0.0) || !std::isfinite(eta))
        return SFG_EINVAL;
    tree->t.stream = (cudaStream_t)stream;
    cudaGetLastError();
    return sfg::sink_timestep(&tree->t, vel, active_idx, n_active, eta, dt, (cudaStream_t)stream);
}

int sfg_set_relative_criterion(sfg_tree *tree, const double *g_prev, double alpha, void *stream)
{
    if (!tree || (g_prev && (!(alpha >= 0.0) || !std::isfinite(alpha)))) return SFG_EINVAL;
    tree->t.stream = (cudaStream_t)stream;
    cudaGetLastError();
    return sfg::set_relative(&tree->t, g_prev, alpha, (cudaStream_t)stream);
}

int sfg_tidal_timestep(const double *tidal, int64_t n, double eta, double *dt, void *stream)
{
    if (n < 0 || (n > 0 && (!tidal || !dt)) || !(eta > 0.0) || !std::isfinite(eta)) return SFG_EINVAL;
    cudaGetLastError();
    return sfg::tidal_timestep(tidal, n, eta, dt, (cudaStream_t)stream);
}

int sfg_hermite_step(const double *pos, const double *vel, const double *mass, const double *soft, int64_t n,
                     const sfg_params *params, double dt, double *pos_out, double *vel_out, void *stream)
{
    if (!pos || !vel || !mass || !soft || !pos_out || !vel_out || n <= 0 || n >= 0x7fffffffLL ||
        !std::isfinite(dt))
        return SFG_EINVAL;
    cudaGetLastError();
    cudaStream_t s = (cudaStream_t)stream;
    const size_t b3 = sizeof(double) * 3 * (size_t)n;
    char *buf = nullptr;
    if (cudaMallocAsync((void **)&buf, 6 * b3 + (size_t)n, s) != cudaSuccess) {
        cudaGetLastError();
        return SFG_ENOMEM;
    }
    double *a0 = (double *)buf, *j0 = a0 + 3 * n, *a1 = j0 + 3 * n, *j1 = a1 + 3 * n, *xp = j1 + 3 * n,
           *vp = xp + 3 * n;
    uint8_t *ones = (uint8_t *)(vp + 3 * n);
    const int64_t n3 = 3 * n;
    const int BT = 256, grid = (int)std::min<int64_t>((n3 + BT - 1) / BT, 4096);
    int rc = cudaMemsetAsync(ones, 1, (size_t)n, s) == cudaSuccess ? SFG_OK : cuda_fail(cudaGetLastError());
    if (rc == SFG_OK) rc = sink_pass(pos, vel, mass, soft, ones, n, params, s, a0, j0);
    if (rc == SFG_OK) {
        k_hermite_predict<<<grid, BT, 0, s>>>(n3, dt, pos, vel, a0, j0, xp, vp);
        rc = sink_pass(xp, vp, mass, soft, ones, n, params, s, a1, j1);
    }
    if (rc == SFG_OK) {
        k_hermite_correct<<<grid, BT, 0, s>>>(n3, dt, pos, vel, a0, j0, a1, j1, pos_out, vel_out);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e);
    }
    cudaFreeAsync(buf, s);
    return rc;
}

int sfg_accel_vjp(sfg_tree *tree, const int64_t *active_idx, int64_t n_active, const double *cot_a,
                  const double *cot_phi, double *d_pos, double *d_mass, void *stream)
{
    if (!tree || n_active < 0 || !d_pos || !d_mass || (n_active > 0 && !cot_a)) return SFG_EINVAL;
    tree->t.stream = (cudaStream_t)stream;
    cudaGetLastError();
    return sfg::accel_vjp(&tree->t, active_idx, n_active, cot_a, cot_phi, d_pos, d_mass, (cudaStream_t)stream);
}

int sfg_get_stats(sfg_tree *tree, sfg_stats *out)
{
    if (!tree || !out) return SFG_EINVAL;
    Tree *t = &tree->t;
    unsigned long long c[NCOUNTERS];
    SFG_CUDA_OK(cudaMemcpyAsync(c, t->d_counters, sizeof(c), cudaMemcpyDeviceToHost, t->stream));
    SFG_CUDA_OK(cudaStreamSynchronize(t->stream));
    sfg_stats s;
    memset(&s, 0, sizeof(s));
    s.n = t->n;
    s.n_nodes = t->nn;
    s.depth = t->depth;
    s.n_levels = t->n_levels;
    for (int a = 0; a < 3; a++) s.x0[a] = t->frame_h.x0[a];
    s.L0 = t->frame_h.L0;
    s.n_p2p = (int64_t)c[0];
    s.n_p2m = (int64_t)c[1];
    s.n_p2p_newton = (int64_t)c[8];
    s.n_overflow = (int64_t)c[2];
    s.n_clouds = t->nclouds;
    s.n_groups = (int64_t)(*(int *)&c[5]);
    s.n_targets = (int64_t)c[6];
    s.n_launches = t->n_launch;
    s.list_walks = t->list_walks;
    float *ms[5] = {&s.build_ms, &s.fwd_ms, &s.fwd_walk_ms, &s.vjp_ms, &s.vjp_walk_ms};
    for (int ph = 0; ph < 5; ph++) {
        *ms[ph] = 0.f;
        if (t->ev_used[ph] && cudaEventElapsedTime(ms[ph], t->ev[2 * ph], t->ev[2 * ph + 1]) != cudaSuccess) {
            cudaGetLastError();
            *ms[ph] = 0.f;
        }
    }
    *out = s;
    return SFG_OK;
}

int sfg_cloud_times(sfg_tree *tree, float *fwd_ms, float *vjp_ms)
{
    if (!tree) return SFG_EINVAL;
    Tree *t = &tree->t;
    const int C = t->nclouds;
    std::vector<unsigned long long> h(2 * (size_t)(C + 1), 0ull);
    if (t->d_ctime) {
        SFG_CUDA_OK(cudaMemcpyAsync(h.data(), t->d_ctime, sizeof(unsigned long long) * h.size(),
                                    cudaMemcpyDeviceToHost, t->stream));
        SFG_CUDA_OK(cudaStreamSynchronize(t->stream));
    }
    float *dst[2] = {fwd_ms, vjp_ms};
    for (int w = 0; w < 2; w++) {
        if (!dst[w]) continue;
        const unsigned long long *c = h.data() + (size_t)w * (C + 1);
        for (int k = 0; k < C; k++)
            dst[w][k] = (t->ctime_used[w] && c[k] > c[C]) ? (float)((double)(c[k] - c[C]) * 1e-6) : 0.f;
    }
    return SFG_OK;
}

int sfg_set_group_share(sfg_tree *tree, int rank, int world)
{
    if (!tree || world < 1 || world > 65536 || rank < 0 || rank >= world) return SFG_EINVAL;
    tree->t.share_rank = rank;
    tree->t.share_world = world;
    return SFG_OK;
}

int sfg_set_timing(sfg_tree *tree, int on)
{
    if (!tree) return SFG_EINVAL;
    tree->t.timing = on != 0;
    return SFG_OK;
}

int sfg_get_status(sfg_tree *tree)
{
    if (!tree) return SFG_EINVAL;
    Tree *t = &tree->t;
    int st = 0;
    SFG_CUDA_OK(cudaMemcpyAsync(&st, t->d_status, sizeof(int), cudaMemcpyDeviceToHost, t->stream));
    SFG_CUDA_OK(cudaStreamSynchronize(t->stream));
    if (st) cudaMemsetAsync(t->d_status, 0, sizeof(int), t->stream);
    if (st & ST_EINVAL) return SFG_EINVAL;
    if (st & ST_EOVERFLOW) return SFG_EOVERFLOW;
    if (st & ST_ETIMEOUT) return SFG_ETIMEOUT;
    return SFG_OK;
}

void sfg_free(sfg_tree *tree)
{
    if (tree) release(tree);
}

int sfg_export(sfg_tree *tree, int field, void *host_dst, size_t bytes)
{
    if (!tree || !host_dst) return SFG_EINVAL;
    Tree *t = &tree->t;
    cudaStream_t s = t->stream;
    const size_t n = (size_t)t->n, nn = (size_t)t->nn;
    SFG_CUDA_OK(cudaStreamSynchronize(s));
    switch (field) {
    case SFG_FIELD_KEYS:
        if (bytes != 8 * n) return SFG_EINVAL;
        SFG_CUDA_OK(cudaMemcpy(host_dst, t->key, bytes, cudaMemcpyDeviceToHost));
        return SFG_OK;
    case SFG_FIELD_ORDER:
        if (bytes != 4 * n) return SFG_EINVAL;
        SFG_CUDA_OK(cudaMemcpy(host_dst, t->order, bytes, cudaMemcpyDeviceToHost));
        return SFG_OK;
    case SFG_FIELD_NODE_HQ:
        if (bytes != 8 * nn) return SFG_EINVAL;
        SFG_CUDA_OK(cudaMemcpy(host_dst, t->Whq, bytes, cudaMemcpyDeviceToHost));
        return SFG_OK;
    case SFG_FIELD_NODE_INT: {
        if (bytes != 64 * nn) return SFG_EINVAL;
        std::vector<int32_t> a(7 * nn);
        std::vector<int4> w(3 * nn);
        SFG_CUDA_OK(cudaMemcpy(&a[0], t->nlevel, 4 * nn, cudaMemcpyDeviceToHost));
        SFG_CUDA_OK(cudaMemcpy(&a[nn], t->nfirst, 4 * nn, cudaMemcpyDeviceToHost));
        SFG_CUDA_OK(cudaMemcpy(&a[2 * nn], t->ncount, 4 * nn, cudaMemcpyDeviceToHost));
        SFG_CUDA_OK(cudaMemcpy(&a[3 * nn], t->nparent, 4 * nn, cudaMemcpyDeviceToHost));
        SFG_CUDA_OK(cudaMemcpy(&a[4 * nn], t->nchild_first, 4 * nn, cudaMemcpyDeviceToHost));
        SFG_CUDA_OK(cudaMemcpy(&a[5 * nn], t->nnchild, 4 * nn, cudaMemcpyDeviceToHost));
        SFG_CUDA_OK(cudaMemcpy(&a[6 * nn], t->ncloud, 4 * nn, cudaMemcpyDeviceToHost));
        SFG_CUDA_OK(cudaMemcpy(&w[0], t->W0, 16 * nn, cudaMemcpyDeviceToHost));
        SFG_CUDA_OK(cudaMemcpy(&w[nn], t->W1, 16 * nn, cudaMemcpyDeviceToHost));
        SFG_CUDA_OK(cudaMemcpy(&w[2 * nn], t->W2, 16 * nn, cudaMemcpyDeviceToHost));
        int32_t *o = (int32_t *)host_dst;
        for (size_t i = 0; i < nn; i++) {
            int32_t *r = o + 16 * i;
            for (int k = 0; k < 6; k++) r[k] = a[k * nn + i];
            int4 w0 = w[i], w1 = w[nn + i], w2 = w[2 * nn + i];
            r[6] = w0.x; r[7] = w0.y; r[8] = w0.z;
            r[9] = w1.x; r[10] = w1.y; r[11] = w1.z;
            r[12] = w2.x; r[13] = w2.y; r[14] = w2.z;
            r[15] = a[6 * nn + i];
        }
        return SFG_OK;
    }
    case SFG_FIELD_NODE_F64: {
        if (bytes != 88 * nn) return SFG_EINVAL;
        std::vector<double> M(nn), com(3 * nn), Q(6 * nn), h(nn);
        SFG_CUDA_OK(cudaMemcpy(M.data(), t->nM, 8 * nn, cudaMemcpyDeviceToHost));
        SFG_CUDA_OK(cudaMemcpy(com.data(), t->ncom, 24 * nn, cudaMemcpyDeviceToHost));
        SFG_CUDA_OK(cudaMemcpy(Q.data(), t->nQ, 48 * nn, cudaMemcpyDeviceToHost));
        SFG_CUDA_OK(cudaMemcpy(h.data(), t->nhmax, 8 * nn, cudaMemcpyDeviceToHost));
        double *o = (double *)host_dst;
        for (size_t i = 0; i < nn; i++) {
            double *r = o + 11 * i;
            r[0] = M[i];
            for (int a = 0; a < 3; a++) r[1 + a] = com[3 * i + a];
            for (int k = 0; k < 6; k++) r[4 + k] = Q[6 * i + k];
            r[10] = h[i];
        }
        return SFG_OK;
    }
    case SFG_FIELD_PARTICLE_F32:
        if (bytes != 16 * n) return SFG_EINVAL;
        SFG_CUDA_OK(cudaMemcpy(host_dst, t->pw, bytes, cudaMemcpyDeviceToHost));
        return SFG_OK;
    case SFG_FIELD_NODE_F32: {
        if (bytes != 36 * nn) return SFG_EINVAL;
        std::vector<float4> e(3 * nn);
        SFG_CUDA_OK(cudaMemcpy(&e[0], t->E0, 16 * nn, cudaMemcpyDeviceToHost));
        SFG_CUDA_OK(cudaMemcpy(&e[nn], t->E1, 16 * nn, cudaMemcpyDeviceToHost));
        SFG_CUDA_OK(cudaMemcpy(&e[2 * nn], t->E2, 16 * nn, cudaMemcpyDeviceToHost));
        float *o = (float *)host_dst;
        for (size_t i = 0; i < nn; i++) {
            const float4 a = e[i], b = e[nn + i], c = e[2 * nn + i];
            const float r[9] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x};
            for (int k = 0; k < 9; k++) o[9 * i + k] = r[k];
        }
        return SFG_OK;
    }
    case SFG_FIELD_FRAMES: {
        const size_t C = (size_t)t->nclouds;
        if (bytes != 32 * C) return SFG_EINVAL;
        double *o = (double *)host_dst;
        for (size_t c = 0; c < C; c++) {
            for (int a = 0; a < 3; a++) o[4 * c + a] = t->frames_h[c].x0[a];
            o[4 * c + 3] = t->frames_h[c].L0;
        }
        return SFG_OK;
    }
    default: return SFG_EINVAL;
    }
}

int sfg_debug_lists(sfg_tree *tree, const int64_t *active_idx, int64_t n_active, int64_t *n_groups,
                    int64_t *n_p2m_total, int64_t *n_p2p_total, int64_t *groups, int32_t *p2m, int32_t *p2p,
                    void *stream)
{
    if (!tree || !n_groups || !n_p2m_total || !n_p2p_total || n_active < 0) return SFG_EINVAL;
    tree->t.stream = (cudaStream_t)stream;
    return sfg::debug_lists(&tree->t, active_idx, n_active, n_groups, n_p2m_total, n_p2p_total, groups, p2m, p2p,
                            (cudaStream_t)stream);
}

} // extern "C"
