/*
 * sfg_oracle.c -- plain, slow, CPU FP64 oracle of the STARFORGE self-gravity path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load this library.  It shares no code, header,
 * table or constant generator with the CUDA path.
 *
 * What it computes (Grudic et al. 2021, STARFORGE methods paper, Sec. 2.2):
 *   - the M4 cubic-spline softened pair law (Sec. 2.2.1: adaptive gas
 *     softening S_i = H_i with the SPH compact spline; averaged (symmetrised)
 *     gas-gas kernels; max(S_*, H) for any pair with a sink; Plummer-equivalent
 *     epsilon = h/2.8 fixes Phi(0) = -2.8 G m / h);
 *   - an FP64 direct sum over all pairs;
 *   - an oct-tree (Sec. 2.2) built on a 2^21-per-axis integer grid with
 *     Morton keys, monopole + quadrupole node moments, and the Barnes-Hut
 *     geometric opening rule theta = L / r > Theta (Sec. 2.2), in two forms:
 *       (a) per particle, paper-faithful: FP64 distance from the target to the
 *           node centre of mass, plus "the target is beyond both softening
 *           radii of every member" (the softened region must be summed pair by
 *           pair, Sec. 2.2.1);
 *       (b) per group of <= G targets, the exact integer, conservative form the
 *           GPU path uses (decisions on integer cell boxes; same decisions here);
 *   - the modified 4th-order Hermite step of sink particles (Sec. 2.3,
 *     predictor and corrector) on FP64 direct sinks-only fields and jerks;
 *   - the analytic vector-Jacobian product of the group-form tree with the
 *     interaction lists frozen (tidal tensor of the same softened kernel, Sec. 2.2),
 *     and a frozen-list re-evaluation used for finite differences.
 *
 * Rounding: IEEE round-to-nearest, compiled with -ffp-contract=off; the frame,
 * keys and node moments follow a fixed operation order so that they are
 * bit-reproducible.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define LMAX 21
#define GRID_MAX 2097151u /* 2^21 - 1 */
#define CAP62 4611686018427387904ull /* 2^62 */

/* ------------------------------------------------------------------------ */
/* Kernel of compact support h (M4 cubic spline), per unit G m.             */
/* phi(r) = W(u)/h, a = g(u)/h^3 * (x_j - x_i), u = r/h; Newtonian u >= 1.   */
/* ------------------------------------------------------------------------ */
double sfgo_W(double u)
{
    if (u < 0.5)
        return 16.0 / 3.0 * u * u - 48.0 / 5.0 * u * u * u * u + 32.0 / 5.0 * u * u * u * u * u - 14.0 / 5.0;
    if (u < 1.0)
        return 1.0 / (15.0 * u) + 32.0 / 3.0 * u * u - 16.0 * u * u * u + 48.0 / 5.0 * u * u * u * u
               - 32.0 / 15.0 * u * u * u * u * u - 16.0 / 5.0;
    return -1.0 / u;
}

double sfgo_g(double u)
{
    if (u < 0.5)
        return 32.0 / 3.0 - 192.0 / 5.0 * u * u + 32.0 * u * u * u;
    if (u < 1.0)
        return 64.0 / 3.0 - 48.0 * u + 192.0 / 5.0 * u * u - 32.0 / 3.0 * u * u * u - 1.0 / (15.0 * u * u * u);
    return 1.0 / (u * u * u);
}

/* g'(u)/u, finite at u = 0. */
double sfgo_dg_over_u(double u)
{
    if (u < 0.5)
        return -384.0 / 5.0 + 96.0 * u;
    if (u < 1.0)
        return -48.0 / u + 384.0 / 5.0 - 32.0 * u + 1.0 / (5.0 * u * u * u * u * u);
    return -3.0 / (u * u * u * u * u);
}

/* One kernel of support h at separation r: a = K d, phi = P, dK/dr / r = Kr. */
static void kernel_one(double r, double h, double *K, double *P, double *Kr)
{
    if (r >= h) {
        *K = 1.0 / (r * r * r);
        *P = -1.0 / r;
        *Kr = -3.0 / (r * r * r * r * r);
    } else {
        double u = r / h;
        *K = sfgo_g(u) / (h * h * h);
        *P = sfgo_W(u) / h;
        *Kr = sfgo_dg_over_u(u) / (h * h * h * h * h);
    }
}

/* Pair rule (Sec. 2.2.1): gas-gas averages the two kernels (symmetrised);
 * a pair with a sink uses one kernel of support max(h_i, h_j). */
static void pair_law(double r, double hi, double hj, int si, int sj, double *K, double *P, double *Kr)
{
    if (si || sj) {
        kernel_one(r, hi > hj ? hi : hj, K, P, Kr);
    } else {
        double K1, P1, R1, K2, P2, R2;
        kernel_one(r, hi, &K1, &P1, &R1);
        kernel_one(r, hj, &K2, &P2, &R2);
        *K = 0.5 * (K1 + K2);
        *P = 0.5 * (P1 + P2);
        *Kr = 0.5 * (R1 + R2);
    }
}

/* Exported for tests: acceleration coefficient and potential of one pair. */
void sfgo_pair(double r, double hi, double hj, int si, int sj, double *out3)
{
    pair_law(r, hi, hj, si, sj, &out3[0], &out3[1], &out3[2]);
}

/* ------------------------------------------------------------------------ */
/* Direct sum: a_i = G sum_{j != i} m_j K_ij (x_j - x_i), phi_i = G sum m_j P_ij */
/* ------------------------------------------------------------------------ */
void sfgo_direct(int64_t n, const double *pos, const double *mass, const double *soft, const uint8_t *sink,
                 double G, int64_t nt, const int64_t *targets, double *acc, double *phi)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i = targets[t];
        double ax = 0, ay = 0, az = 0, p = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i)
                continue;
            double dx = pos[3 * j] - pos[3 * i], dy = pos[3 * j + 1] - pos[3 * i + 1], dz = pos[3 * j + 2] - pos[3 * i + 2];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            double K, P, Kr;
            pair_law(r, soft[i], soft[j], sink ? sink[i] : 0, sink ? sink[j] : 0, &K, &P, &Kr);
            ax += mass[j] * K * dx;
            ay += mass[j] * K * dy;
            az += mass[j] * K * dz;
            p += mass[j] * P;
        }
        acc[3 * t] = G * ax;
        acc[3 * t + 1] = G * ay;
        acc[3 * t + 2] = G * az;
        phi[t] = G * p;
    }
}

/* One pair's tidal term (per unit G m_j): T += -[K I + (dK/dr / r) d d^T],
 * d = x_j - x_i: the derivative of a = m K(r) d with respect to x_i (Sec. 2.2
 * defines T = -grad grad Phi; Sec. 2.2.1 sums it with the same softened kernel
 * and symmetrisation as g).  Components xx yy zz xy xz yz. */
static void pair_tidal(double m, double K, double Kr, double dx, double dy, double dz, double T[6])
{
    T[0] -= m * (K + Kr * dx * dx);
    T[1] -= m * (K + Kr * dy * dy);
    T[2] -= m * (K + Kr * dz * dz);
    T[3] -= m * Kr * dx * dy;
    T[4] -= m * Kr * dx * dz;
    T[5] -= m * Kr * dy * dz;
}

/* Direct-sum tidal tensor at the targets (all pairs j != i). */
void sfgo_direct_tidal(int64_t n, const double *pos, const double *mass, const double *soft, const uint8_t *sink,
                       double G, int64_t nt, const int64_t *targets, double *tidal)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i = targets[t];
        double T[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t j = 0; j < n; j++) {
            if (j == i)
                continue;
            double dx = pos[3 * j] - pos[3 * i], dy = pos[3 * j + 1] - pos[3 * i + 1], dz = pos[3 * j + 2] - pos[3 * i + 2];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            double K, P, Kr;
            pair_law(r, soft[i], soft[j], sink ? sink[i] : 0, sink ? sink[j] : 0, &K, &P, &Kr);
            pair_tidal(mass[j], K, Kr, dx, dy, dz, T);
        }
        for (int c = 0; c < 6; c++) tidal[6 * t + c] = G * T[c];
    }
}

/* One pair's jerk term (per unit G m_j): the time derivative of a = m K(r) d
 * along the motion, d = x_j - x_i, w = v_j - v_i:
 *   j += K w + (dK/dr / r) (d . w) d
 * (Sec. 2.2: j in the same pass as g, with spatial derivatives of the same
 * softened kernel and symmetrisation, Sec. 2.2.1). */
static void pair_jerk(double m, double K, double Kr, const double d[3], const double w[3], double j[3])
{
    double dw = d[0] * w[0] + d[1] * w[1] + d[2] * w[2];
    for (int a = 0; a < 3; a++) j[a] += m * (K * w[a] + Kr * dw * d[a]);
}

/* Direct-sum jerk at the targets (all pairs j != i), vel [n][3]. */
void sfgo_direct_jerk(int64_t n, const double *pos, const double *vel, const double *mass, const double *soft,
                      const uint8_t *sink, double G, int64_t nt, const int64_t *targets, double *jerk)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i = targets[t];
        double J[3] = {0, 0, 0};
        for (int64_t k = 0; k < n; k++) {
            if (k == i)
                continue;
            double d[3], w[3];
            for (int a = 0; a < 3; a++) {
                d[a] = pos[3 * k + a] - pos[3 * i + a];
                w[a] = vel[3 * k + a] - vel[3 * i + a];
            }
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double K, P, Kr;
            pair_law(r, soft[i], soft[k], sink ? sink[i] : 0, sink ? sink[k] : 0, &K, &P, &Kr);
            pair_jerk(mass[k], K, Kr, d, w, J);
        }
        for (int a = 0; a < 3; a++) jerk[3 * t + a] = G * J[a];
    }
}

/* Field and jerk of every particle from every other, all treated as sinks
 * (the sinks-only pass of Sec. 2.3, summed directly in FP64). */
static void sink_field_jerk(int64_t n, const double *pos, const double *vel, const double *mass, const double *soft,
                            double G, double *acc, double *jerk)
{
    for (int64_t i = 0; i < n; i++) {
        double A[3] = {0, 0, 0}, J[3] = {0, 0, 0};
        for (int64_t k = 0; k < n; k++) {
            if (k == i)
                continue;
            double d[3], w[3];
            for (int a = 0; a < 3; a++) {
                d[a] = pos[3 * k + a] - pos[3 * i + a];
                w[a] = vel[3 * k + a] - vel[3 * i + a];
            }
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double K, P, Kr;
            pair_law(r, soft[i], soft[k], 1, 1, &K, &P, &Kr);
            for (int a = 0; a < 3; a++) A[a] += mass[k] * K * d[a];
            pair_jerk(mass[k], K, Kr, d, w, J);
        }
        for (int a = 0; a < 3; a++) {
            acc[3 * i + a] = G * A[a];
            jerk[3 * i + a] = G * J[a];
        }
    }
}

/* One step of the modified 4th-order Hermite integrator for sink particles
 * (Sec. 2.3, the predictor and corrector equations).  The field a0 and jerk
 * j0 are evaluated at the start (x0, v0); the prediction is
 *   x_p = x0 + dt v0 + dt^2/2 a0 + dt^3/6 j0,   v_p = v0 + dt a0 + dt^2/2 j0;
 * the field and jerk are evaluated again at (x_p, v_p), giving a1, j1; the
 * correction updates the velocity first and the position from it:
 *   v1 = v0 + dt/2 (a1 + a0) + dt^2/12 (j0 - j1),
 *   x1 = x0 + dt/2 (v1 + v0) + dt^2/12 (a0 - a1).
 * pos, vel [n][3] (the start), pos1, vel1 [n][3] (the end). */
void sfgo_hermite_step(int64_t n, const double *pos, const double *vel, const double *mass, const double *soft,
                       double G, double dt, double *pos1, double *vel1)
{
    size_t b = sizeof(double) * 3 * (size_t)(n > 0 ? n : 1);
    double *a0 = malloc(b), *j0 = malloc(b), *a1 = malloc(b), *j1 = malloc(b), *xp = malloc(b), *vp = malloc(b);
    sink_field_jerk(n, pos, vel, mass, soft, G, a0, j0);
    for (int64_t q = 0; q < 3 * n; q++) {
        xp[q] = pos[q] + dt * vel[q] + (dt * dt / 2.0) * a0[q] + (dt * dt * dt / 6.0) * j0[q];
        vp[q] = vel[q] + dt * a0[q] + (dt * dt / 2.0) * j0[q];
    }
    sink_field_jerk(n, xp, vp, mass, soft, G, a1, j1);
    for (int64_t q = 0; q < 3 * n; q++) {
        vel1[q] = vel[q] + (dt / 2.0) * (a1[q] + a0[q]) + (dt * dt / 12.0) * (j0[q] - j1[q]);
        pos1[q] = pos[q] + (dt / 2.0) * (vel1[q] + vel[q]) + (dt * dt / 12.0) * (a0[q] - a1[q]);
    }
    free(a0);
    free(j0);
    free(a1);
    free(j1);
    free(xp);
    free(vp);
}

/* Tidal timestep of Sec. 2.3, Eq. for Delta t_tidal: sqrt(eta) (|T|^2 / 6)^(-1/4)
 * with |T| the Frobenius norm (T given as xx yy zz xy xz yz); infinite when T = 0. */
void sfgo_tidal_dt(int64_t n, const double *tidal, double eta, double *dt)
{
    for (int64_t i = 0; i < n; i++) {
        const double *T = tidal + 6 * i;
        double f2 = T[0] * T[0] + T[1] * T[1] + T[2] * T[2] + 2.0 * (T[3] * T[3] + T[4] * T[4] + T[5] * T[5]);
        dt[i] = f2 > 0.0 ? sqrt(eta) * pow(f2 / 6.0, -0.25) : HUGE_VAL;
    }
}

/* ------------------------------------------------------------------------ */
/* Tree                                                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t level;
    int64_t first, count, parent, child_first;
    int32_t nchild;
    uint32_t corner[3]; /* cell corner, level-21 grid units */
    uint32_t lo[3], hi[3]; /* integer box of member cells, inclusive */
    uint32_t cq[3];        /* grid cell of the centre of mass */
    uint64_t hq;           /* ceil((hmax / cell)^2), capped at 2^62 */
    double M, com[3], Q[6]; /* Q: xx yy zz xy xz yz, traceless, about com */
    double S[6];            /* second moment sum m d d^T about com (xx yy zz xy xz yz) */
    double hmax, flo[3], fhi[3]; /* max softening; FP64 tight box */
} onode;

typedef struct {
    int64_t node, tfirst, tcount; /* targets: tgt[tfirst .. tfirst+tcount) (sorted ranks) */
    uint32_t lo[3], hi[3];
    uint64_t hq;
    double gmin; /* smallest |g_prev| of the targets (relative criterion) */
    int walked;
    int64_t n_p2m, n_p2p;
    int64_t *p2m, *p2p; /* accepted nodes; opened leaves */
} ogroup;

typedef struct sfgo_tree {
    int64_t n;
    int leaf_size;
    double x0[3], L0, scale;
    double *pos, *mass, *soft; /* sorted */
    uint8_t *sink;
    int64_t *order, *rank;
    uint64_t *key;
    uint32_t *q;
    int64_t nn;
    onode *nodes;
    /* last group walk */
    int gsize;
    double theta;
    int64_t ng;
    ogroup *groups;
    int64_t *tgt;       /* unique active sorted ranks, grouped */
    int64_t *tgroup;    /* sorted rank -> group id (-1) */
    /* relative (acceleration-based) opening criterion, off when gprev == NULL */
    double *gprev;      /* |g| of the previous step per sorted rank */
    double alpha, Grel; /* error tolerance; G multiplying node masses */
} sfgo_tree;

/* Frame: per-axis min; root side L0 = smallest power of two >= largest extent. */
static void make_frame(int64_t n, const double *pos, double x0[3], double *L0)
{
    double lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
        lo[a] = pos[a];
        hi[a] = pos[a];
    }
    for (int64_t i = 0; i < n; i++)
        for (int a = 0; a < 3; a++) {
            double v = pos[3 * i + a];
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
    double E = 0.0;
    for (int a = 0; a < 3; a++) {
        x0[a] = lo[a];
        double e = hi[a] - lo[a];
        if (e > E) E = e;
    }
    if (E == 0.0) {
        *L0 = 1.0;
    } else {
        int ex;
        double f = frexp(E, &ex);
        *L0 = (f == 0.5) ? E : ldexp(1.0, ex);
    }
}

/* Integer cell of a coordinate: floor((x - x0) * 2^21 / L0), clamped. */
static uint32_t cell_of(double x, double x0, double scale)
{
    double s = (x - x0) * scale;
    if (!(s > 0.0)) return 0u;
    if (s >= 2097152.0) return GRID_MAX;
    return (uint32_t)s;
}

static uint64_t morton(uint32_t qx, uint32_t qy, uint32_t qz)
{
    uint64_t k = 0;
    for (int b = 0; b < LMAX; b++) {
        k |= (uint64_t)((qx >> b) & 1u) << (3 * b + 2);
        k |= (uint64_t)((qy >> b) & 1u) << (3 * b + 1);
        k |= (uint64_t)((qz >> b) & 1u) << (3 * b);
    }
    return k;
}

static uint64_t hq_of(double h, double scale)
{
    double v = h * scale;
    double v2 = v * v;
    if (!(v2 < 4611686018427387904.0)) return CAP62;
    uint64_t c = (uint64_t)ceil(v2);
    return c > 0 ? c : 1u; /* >= 1: a node touching a target's cell is always opened */
}

typedef struct { uint64_t key; int64_t idx; } kv;
static int kv_cmp(const void *a, const void *b)
{
    const kv *x = (const kv *)a, *y = (const kv *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

static void node_centre(const sfgo_tree *t, const onode *nd, double c[3])
{
    double half_cell = ldexp(t->L0, -22);
    for (int a = 0; a < 3; a++)
        c[a] = t->x0[a] + (double)(2u * nd->corner[a] + (1u << (LMAX - nd->level))) * half_cell;
}

/* Moments of every node (Sec. 2.2: mass, centre of mass, and the traceless
 * quadrupole Q = sum m (3 d d^T - |d|^2 I) about the centre of mass, d =
 * x - com).  Every node first sums about its own cell centre c: the mass M,
 * the first moment s = sum m (x - c) and the second moment S' = sum m (x - c)
 * (x - c)^T -- over its members in sorted order for a leaf, over its
 * children in octant order for an internal node, each child entering with its
 * mass at its centre of mass plus its own second moment about it.  Then the
 * parallel-axis theorem moves S' to the centre of mass: com = c + s/M and
 * S = S' - s (s/M)^T, and Q = 3 S - tr(S) I.  A massless node keeps com = c.
 * Fixed operation order; the products added into S' and the shift use an
 * explicit fused multiply-add (one rounding, C99 fma), everything else is
 * plain IEEE add/mul/div without contraction. */
static void compute_moments(sfgo_tree *t, const double *pos, const double *mass)
{
    for (int64_t i = t->nn - 1; i >= 0; i--) {
        onode *nd = &t->nodes[i];
        double c[3];
        node_centre(t, nd, c);
        double M = 0.0, s[3] = {0.0, 0.0, 0.0}, S[6] = {0, 0, 0, 0, 0, 0};
        if (nd->nchild == 0) {
            for (int64_t k = nd->first; k < nd->first + nd->count; k++) {
                double m = mass[k];
                double d[3], md[3];
                for (int a = 0; a < 3; a++) d[a] = pos[3 * k + a] - c[a];
                M = M + m;
                for (int a = 0; a < 3; a++) md[a] = m * d[a];
                for (int a = 0; a < 3; a++) s[a] = s[a] + md[a];
                S[0] = fma(md[0], d[0], S[0]);
                S[1] = fma(md[1], d[1], S[1]);
                S[2] = fma(md[2], d[2], S[2]);
                S[3] = fma(md[0], d[1], S[3]);
                S[4] = fma(md[0], d[2], S[4]);
                S[5] = fma(md[1], d[2], S[5]);
            }
        } else {
            for (int q = 0; q < nd->nchild; q++) {
                const onode *ch = &t->nodes[nd->child_first + q];
                double d[3], md[3];
                for (int a = 0; a < 3; a++) d[a] = ch->com[a] - c[a];
                M = M + ch->M;
                for (int a = 0; a < 3; a++) md[a] = ch->M * d[a];
                for (int a = 0; a < 3; a++) s[a] = s[a] + md[a];
                S[0] = S[0] + fma(md[0], d[0], ch->S[0]);
                S[1] = S[1] + fma(md[1], d[1], ch->S[1]);
                S[2] = S[2] + fma(md[2], d[2], ch->S[2]);
                S[3] = S[3] + fma(md[0], d[1], ch->S[3]);
                S[4] = S[4] + fma(md[0], d[2], ch->S[4]);
                S[5] = S[5] + fma(md[1], d[2], ch->S[5]);
            }
        }
        if (M > 0.0) {
            double dl[3];
            for (int a = 0; a < 3; a++) {
                dl[a] = s[a] / M;
                nd->com[a] = c[a] + dl[a];
            }
            S[0] = fma(-s[0], dl[0], S[0]);
            S[1] = fma(-s[1], dl[1], S[1]);
            S[2] = fma(-s[2], dl[2], S[2]);
            S[3] = fma(-s[0], dl[1], S[3]);
            S[4] = fma(-s[0], dl[2], S[4]);
            S[5] = fma(-s[1], dl[2], S[5]);
        } else {
            for (int a = 0; a < 3; a++) nd->com[a] = c[a];
        }
        double tr = S[0] + S[1] + S[2];
        nd->M = M;
        for (int q = 0; q < 6; q++) nd->S[q] = S[q];
        nd->Q[0] = 3.0 * S[0] - tr;
        nd->Q[1] = 3.0 * S[1] - tr;
        nd->Q[2] = 3.0 * S[2] - tr;
        nd->Q[3] = 3.0 * S[3];
        nd->Q[4] = 3.0 * S[4];
        nd->Q[5] = 3.0 * S[5];
    }
}

/* Geometry that does not depend on the moments' values except cq. */
static void compute_geometry(sfgo_tree *t)
{
    for (int64_t i = t->nn - 1; i >= 0; i--) {
        onode *nd = &t->nodes[i];
        double hmax = 0.0;
        for (int a = 0; a < 3; a++) {
            nd->lo[a] = GRID_MAX;
            nd->hi[a] = 0;
            nd->flo[a] = INFINITY;
            nd->fhi[a] = -INFINITY;
        }
        for (int64_t k = nd->first; k < nd->first + nd->count; k++) {
            for (int a = 0; a < 3; a++) {
                uint32_t qa = t->q[3 * k + a];
                if (qa < nd->lo[a]) nd->lo[a] = qa;
                if (qa > nd->hi[a]) nd->hi[a] = qa;
                double v = t->pos[3 * k + a];
                if (v < nd->flo[a]) nd->flo[a] = v;
                if (v > nd->fhi[a]) nd->fhi[a] = v;
            }
            if (t->soft[k] > hmax) hmax = t->soft[k];
        }
        nd->hmax = hmax;
        nd->hq = hq_of(hmax, t->scale);
        for (int a = 0; a < 3; a++) nd->cq[a] = cell_of(nd->com[a], t->x0[a], t->scale);
    }
}

sfgo_tree *sfgo_build(int64_t n, const double *pos, const double *mass, const double *soft, const uint8_t *sink,
                      int leaf_size)
{
    if (n <= 0 || leaf_size < 1) return NULL;
    sfgo_tree *t = (sfgo_tree *)calloc(1, sizeof(sfgo_tree));
    t->n = n;
    t->leaf_size = leaf_size;
    make_frame(n, pos, t->x0, &t->L0);
    t->scale = ldexp(1.0, LMAX) / t->L0;

    /* keys, stable sort by (key, original index) */
    kv *arr = (kv *)malloc(sizeof(kv) * n);
    for (int64_t i = 0; i < n; i++) {
        uint32_t qx = cell_of(pos[3 * i], t->x0[0], t->scale);
        uint32_t qy = cell_of(pos[3 * i + 1], t->x0[1], t->scale);
        uint32_t qz = cell_of(pos[3 * i + 2], t->x0[2], t->scale);
        arr[i].key = morton(qx, qy, qz);
        arr[i].idx = i;
    }
    qsort(arr, (size_t)n, sizeof(kv), kv_cmp);
    t->key = (uint64_t *)malloc(8 * n);
    t->order = (int64_t *)malloc(8 * n);
    t->rank = (int64_t *)malloc(8 * n);
    t->pos = (double *)malloc(24 * n);
    t->mass = (double *)malloc(8 * n);
    t->soft = (double *)malloc(8 * n);
    t->sink = (uint8_t *)malloc(n);
    t->q = (uint32_t *)malloc(12 * n);
    for (int64_t r = 0; r < n; r++) {
        int64_t i = arr[r].idx;
        t->key[r] = arr[r].key;
        t->order[r] = i;
        t->rank[i] = r;
        for (int a = 0; a < 3; a++) {
            t->pos[3 * r + a] = pos[3 * i + a];
            t->q[3 * r + a] = cell_of(pos[3 * i + a], t->x0[a], t->scale);
        }
        t->mass[r] = mass[i];
        t->soft[r] = soft[i];
        t->sink[r] = sink ? sink[i] : 0;
    }
    free(arr);

    /* octree, breadth-first: node ids ordered by (level, first sorted index) */
    int64_t cap = 1024;
    t->nodes = (onode *)calloc(cap, sizeof(onode));
    t->nodes[0].level = 0;
    t->nodes[0].first = 0;
    t->nodes[0].count = n;
    t->nodes[0].parent = -1;
    t->nn = 1;
    for (int64_t i = 0; i < t->nn; i++) {
        onode nd = t->nodes[i];
        for (int a = 0; a < 3; a++) t->nodes[i].corner[a] = (t->q[3 * nd.first + a] >> (LMAX - nd.level)) << (LMAX - nd.level);
        if (nd.count <= leaf_size || nd.level == LMAX) {
            t->nodes[i].child_first = -1;
            t->nodes[i].nchild = 0;
            continue;
        }
        int cshift = 3 * (LMAX - nd.level - 1);
        t->nodes[i].child_first = t->nn;
        int64_t start = nd.first, end = nd.first + nd.count;
        for (int64_t k = nd.first + 1; k <= end; k++) {
            if (k == end || ((t->key[k] >> cshift) & 7u) != ((t->key[start] >> cshift) & 7u)) {
                if (t->nn == cap) {
                    cap *= 2;
                    t->nodes = (onode *)realloc(t->nodes, sizeof(onode) * cap);
                }
                onode *c = &t->nodes[t->nn++];
                memset(c, 0, sizeof(onode));
                c->level = nd.level + 1;
                c->first = start;
                c->count = k - start;
                c->parent = i;
                start = k;
            }
        }
        t->nodes[i].nchild = (int32_t)(t->nn - t->nodes[i].child_first);
    }
    compute_moments(t, t->pos, t->mass);
    compute_geometry(t);
    return t;
}

static void free_walk(sfgo_tree *t)
{
    if (t->groups) {
        for (int64_t g = 0; g < t->ng; g++) {
            free(t->groups[g].p2m);
            free(t->groups[g].p2p);
        }
    }
    free(t->groups);
    free(t->tgt);
    free(t->tgroup);
    t->groups = NULL;
    t->tgt = NULL;
    t->tgroup = NULL;
    t->ng = 0;
}

void sfgo_free(sfgo_tree *t)
{
    if (!t) return;
    free_walk(t);
    free(t->pos); free(t->mass); free(t->soft); free(t->sink); free(t->gprev);
    free(t->order); free(t->rank); free(t->key); free(t->q); free(t->nodes);
    free(t);
}

void sfgo_info(const sfgo_tree *t, double *frame4, int64_t *nn)
{
    for (int a = 0; a < 3; a++) frame4[a] = t->x0[a];
    frame4[3] = t->L0;
    *nn = t->nn;
}

void sfgo_keys(const sfgo_tree *t, uint64_t *key_sorted, int64_t *order)
{
    memcpy(key_sorted, t->key, 8 * t->n);
    memcpy(order, t->order, 8 * t->n);
}

/* per node: level first count parent child_first nchild corner[3] lo[3] hi[3] cq[3] hq  (19 int64) */
void sfgo_nodes_int(const sfgo_tree *t, int64_t *out)
{
    for (int64_t i = 0; i < t->nn; i++) {
        const onode *nd = &t->nodes[i];
        int64_t *o = out + 19 * i;
        o[0] = nd->level; o[1] = nd->first; o[2] = nd->count; o[3] = nd->parent;
        o[4] = nd->child_first; o[5] = nd->nchild;
        for (int a = 0; a < 3; a++) {
            o[6 + a] = nd->corner[a];
            o[9 + a] = nd->lo[a];
            o[12 + a] = nd->hi[a];
            o[15 + a] = nd->cq[a];
        }
        o[18] = (int64_t)nd->hq;
    }
}

/* per node: M com[3] Q[6] hmax flo[3] fhi[3]  (17 doubles) */
void sfgo_nodes_f64(const sfgo_tree *t, double *out)
{
    for (int64_t i = 0; i < t->nn; i++) {
        const onode *nd = &t->nodes[i];
        double *o = out + 17 * i;
        o[0] = nd->M;
        for (int a = 0; a < 3; a++) o[1 + a] = nd->com[a];
        for (int c = 0; c < 6; c++) o[4 + c] = nd->Q[c];
        o[10] = nd->hmax;
        for (int a = 0; a < 3; a++) {
            o[11 + a] = nd->flo[a];
            o[14 + a] = nd->fhi[a];
        }
    }
}

/* ---------------- group form: integer, conservative opening rule --------- */
/* The group level of a cloud holding U targets: the largest L with
 * G 8^L <= U (0 below 8 G), the depth at which a uniform cloud's nodes hold
 * about G targets.  Nodes above it are always opened and their children are
 * not packed together, so that no group spans sparse octants of the top
 * levels (such groups had boxes covering much of the cloud). */
static int group_level(int64_t U, int gsize)
{
    int L = 0;
    for (int64_t v = (int64_t)gsize * 8; v <= U && L < 21; v *= 8) L++;
    return L;
}

/* ceil(4^(21-l) / theta^2), capped at 2^62: "open if L/r > theta" with L and
 * r in cell units (L = 2^(21-l) cells). */
static uint64_t open_threshold(int level, double theta)
{
    double v = ldexp(1.0, 2 * (LMAX - level)) / (theta * theta);
    if (!(v < 4611686018427387904.0)) return CAP62;
    return (uint64_t)ceil(v);
}

/* Gap, in cells, between the cell intervals [alo, ahi+1] and [blo, bhi+1]. */
static uint64_t cell_gap(uint32_t alo, uint32_t ahi, uint32_t blo, uint32_t bhi)
{
    int64_t g1 = (int64_t)blo - (int64_t)ahi - 1;
    int64_t g2 = (int64_t)alo - (int64_t)bhi - 1;
    int64_t g = g1 > g2 ? g1 : g2;
    return g > 0 ? (uint64_t)g : 0u;
}

/* Relative criterion of Sec. 2.2 (the acceleration-based rule the paper takes
 * from GADGET-2, applied together with the geometric one): accept only if the
 * node's quadrupole-order error scale G M L^2 / r^4 is at most alpha |g_prev|.
 * Group form, conservative for every target: r >= sqrt(sc) cells (sc = the
 * squared whole-cell gap of the geometric clause) and |g_prev| >= gmin, so
 * test G M L^2 <= alpha gmin (sc cell^2)^2, as exactly these IEEE products
 * (each rounded once, in this order, no contraction). */
static int accept_relative(const sfgo_tree *t, const ogroup *g, const onode *nd, uint64_t sc)
{
    double L = ldexp(t->L0, -nd->level);
    double cell = ldexp(t->L0, -LMAX);
    double lhs = (t->Grel * nd->M) * (L * L);
    double r2 = (double)sc * (cell * cell);
    double rhs = (t->alpha * g->gmin) * (r2 * r2);
    return lhs <= rhs;
}

static int accept_group(const sfgo_tree *t, const ogroup *g, const onode *nd, const uint64_t *T)
{
    uint64_t sc = 0, sb = 0;
    for (int a = 0; a < 3; a++) {
        uint64_t gc = cell_gap(nd->cq[a], nd->cq[a], g->lo[a], g->hi[a]);
        uint64_t gb = cell_gap(nd->lo[a], nd->hi[a], g->lo[a], g->hi[a]);
        sc += gc * gc;
        sb += gb * gb;
    }
    uint64_t hneed = g->hq > nd->hq ? g->hq : nd->hq;
    if (!(sc >= T[nd->level] && sb >= hneed)) return 0;
    return t->gprev ? accept_relative(t, g, nd, sc) : 1;
}

/* Switch the relative criterion on (g_prev = |g| per particle in the input
 * order, alpha > 0) or off (g_prev == NULL). */
void sfgo_set_relative(sfgo_tree *t, const double *g_prev, double alpha, double G)
{
    free(t->gprev);
    t->gprev = NULL;
    if (!g_prev) return;
    t->gprev = (double *)malloc(8 * t->n);
    for (int64_t r = 0; r < t->n; r++) t->gprev[r] = g_prev[t->order[r]];
    t->alpha = alpha;
    t->Grel = G;
}

typedef struct { int64_t *v; int64_t n, cap; } ivec;
static void ivec_push(ivec *a, int64_t x)
{
    if (a->n == a->cap) {
        a->cap = a->cap ? 2 * a->cap : 64;
        a->v = (int64_t *)realloc(a->v, 8 * a->cap);
    }
    a->v[a->n++] = x;
}

static void walk_group(const sfgo_tree *t, const ogroup *g, int64_t ni, const uint64_t *T, ivec *p2m, ivec *p2p)
{
    const onode *nd = &t->nodes[ni];
    if (accept_group(t, g, nd, T)) {
        ivec_push(p2m, ni);
    } else if (nd->nchild == 0) {
        ivec_push(p2p, ni);
    } else {
        for (int c = 0; c < nd->nchild; c++) walk_group(t, g, nd->child_first + c, T, p2m, p2p);
    }
}

/* Groups of <= G active targets, contiguous in sorted (Morton) order:
 *   - the root, if it holds 1..G targets;
 *   - under every internal node holding more than G targets, its children
 *     that hold 1..G targets are packed greedily, in octant order, into runs
 *     of at most G targets (a child holding more than G is not packed: if it
 *     is internal its own children are packed, if it is a leaf it is cut);
 *   - a leaf holding more than G targets is cut into runs of G.
 * Groups are numbered by their first target (Morton order).  Every group (or,
 * if need != NULL, only the groups holding a listed original index) is then
 * walked from the root.  Returns the number of groups. */
typedef struct { int64_t tfirst, tcount, node; } grun;
static int grun_cmp(const void *a, const void *b)
{
    const grun *x = (const grun *)a, *y = (const grun *)b;
    return (x->tfirst > y->tfirst) - (x->tfirst < y->tfirst);
}

int64_t sfgo_walk(sfgo_tree *t, const int64_t *active, int64_t n_active, int gsize, double theta,
                  const int64_t *need, int64_t n_need)
{
    free_walk(t);
    int64_t n = t->n;
    t->gsize = gsize;
    t->theta = theta;
    uint8_t *act = (uint8_t *)calloc(n, 1);
    for (int64_t k = 0; k < n_active; k++) act[t->rank[active[k]]] = 1;
    int64_t *pre = (int64_t *)malloc(8 * (n + 1));
    pre[0] = 0;
    for (int64_t r = 0; r < n; r++) pre[r + 1] = pre[r] + act[r];
    int64_t U = pre[n];
    t->tgt = (int64_t *)malloc(8 * (U > 0 ? U : 1));
    for (int64_t r = 0, k = 0; r < n; r++)
        if (act[r]) t->tgt[k++] = r;
    t->tgroup = (int64_t *)malloc(8 * n);
    for (int64_t r = 0; r < n; r++) t->tgroup[r] = -1;

    int64_t rcap = 64, nr = 0;
    grun *runs = (grun *)malloc(sizeof(grun) * rcap);
#define EMIT(tf, tc, nd)                                                   \
    do {                                                                   \
        if (nr == rcap) {                                                  \
            rcap *= 2;                                                     \
            runs = (grun *)realloc(runs, sizeof(grun) * rcap);             \
        }                                                                  \
        runs[nr].tfirst = (tf);                                            \
        runs[nr].tcount = (tc);                                            \
        runs[nr].node = (nd);                                              \
        nr++;                                                              \
    } while (0)
    const int glevel = group_level(U, gsize);
    for (int64_t i = 0; i < t->nn; i++) {
        const onode *nd = &t->nodes[i];
        int64_t c = pre[nd->first + nd->count] - pre[nd->first];
        if (c == 0) continue;
        /* a node is opened (its children considered) when it holds more than
         * G targets, or when it lies above the group level and has children */
        const int open = nd->nchild > 0 && (c > gsize || nd->level < glevel);
        if (i == 0 && !open && c <= gsize) EMIT(pre[nd->first], c, i);
        if (c > gsize && nd->nchild == 0 && i == 0)
            for (int64_t s = 0; s < c; s += gsize) EMIT(pre[nd->first] + s, (c - s) < gsize ? (c - s) : gsize, i);
        if (!open) continue;
        /* siblings are packed together only below the group level */
        const int pack = nd->level >= glevel;
        int64_t run_first = -1, run_count = 0;
        for (int k = 0; k < nd->nchild; k++) {
            const onode *ch = &t->nodes[nd->child_first + k];
            int64_t tf = pre[ch->first];
            int64_t cc = pre[ch->first + ch->count] - tf;
            if (cc == 0) continue;
            const int ch_open = ch->nchild > 0 && (cc > gsize || ch->level < glevel);
            if (cc > gsize || ch_open) {
                if (run_count) EMIT(run_first, run_count, i);
                run_count = 0;
                if (ch->nchild == 0)
                    for (int64_t s = 0; s < cc; s += gsize) EMIT(tf + s, (cc - s) < gsize ? (cc - s) : gsize, i);
                continue;
            }
            if (!pack) {
                EMIT(tf, cc, i);
                continue;
            }
            if (run_count + cc > gsize) {
                EMIT(run_first, run_count, i);
                run_count = 0;
            }
            if (run_count == 0) run_first = tf;
            run_count += cc;
        }
        if (run_count) EMIT(run_first, run_count, i);
    }
#undef EMIT
    qsort(runs, (size_t)nr, sizeof(grun), grun_cmp);
    int64_t ng = nr;
    t->groups = (ogroup *)calloc(ng > 0 ? ng : 1, sizeof(ogroup));
    for (int64_t g = 0; g < ng; g++) {
        ogroup *G = &t->groups[g];
        G->node = runs[g].node;
        G->tfirst = runs[g].tfirst;
        G->tcount = runs[g].tcount;
        for (int a = 0; a < 3; a++) {
            G->lo[a] = GRID_MAX;
            G->hi[a] = 0;
        }
        G->hq = 0;
        G->gmin = HUGE_VAL;
        for (int64_t k = G->tfirst; k < G->tfirst + G->tcount; k++) {
            int64_t r = t->tgt[k];
            t->tgroup[r] = g;
            if (t->gprev && t->gprev[r] < G->gmin) G->gmin = t->gprev[r];
            for (int a = 0; a < 3; a++) {
                if (t->q[3 * r + a] < G->lo[a]) G->lo[a] = t->q[3 * r + a];
                if (t->q[3 * r + a] > G->hi[a]) G->hi[a] = t->q[3 * r + a];
            }
            uint64_t h = hq_of(t->soft[r], t->scale);
            if (h > G->hq) G->hq = h;
        }
    }
    free(runs);
    t->ng = ng;
    uint64_t T[LMAX + 1];
    for (int l = 0; l <= LMAX; l++) T[l] = open_threshold(l, theta);
    uint8_t *want = NULL;
    if (need) {
        want = (uint8_t *)calloc(ng > 0 ? ng : 1, 1);
        for (int64_t k = 0; k < n_need; k++) {
            int64_t g = t->tgroup[t->rank[need[k]]];
            if (g >= 0) want[g] = 1;
        }
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t g = 0; g < ng; g++) {
        if (want && !want[g]) continue;
        ivec a = {0, 0, 0}, b = {0, 0, 0};
        walk_group(t, &t->groups[g], 0, T, &a, &b);
        t->groups[g].p2m = a.v;
        t->groups[g].n_p2m = a.n;
        t->groups[g].p2p = b.v;
        t->groups[g].n_p2p = b.n;
        t->groups[g].walked = 1;
    }
    free(want);
    free(act);
    free(pre);
    return ng;
}

/* per group: node tfirst tcount walked n_p2m n_p2p_leaves n_p2p_particles lo[3] hi[3] hq  (14 int64) */
void sfgo_groups(const sfgo_tree *t, int64_t *out)
{
    for (int64_t g = 0; g < t->ng; g++) {
        const ogroup *G = &t->groups[g];
        int64_t *o = out + 14 * g;
        int64_t np = 0;
        for (int64_t k = 0; k < G->n_p2p; k++) np += t->nodes[G->p2p[k]].count;
        o[0] = G->node; o[1] = G->tfirst; o[2] = G->tcount; o[3] = G->walked;
        o[4] = G->n_p2m; o[5] = G->n_p2p; o[6] = np;
        for (int a = 0; a < 3; a++) {
            o[7 + a] = G->lo[a];
            o[10 + a] = G->hi[a];
        }
        o[13] = (int64_t)G->hq;
    }
}

void sfgo_group_targets(const sfgo_tree *t, int64_t *out)
{
    int64_t nt = 0;
    for (int64_t g = 0; g < t->ng; g++) nt += t->groups[g].tcount;
    memcpy(out, t->tgt, 8 * nt);
}

/* Lists of one group (sizes from sfgo_groups). */
void sfgo_group_lists(const sfgo_tree *t, int64_t g, int64_t *p2m, int64_t *p2p)
{
    const ogroup *G = &t->groups[g];
    if (G->n_p2m) memcpy(p2m, G->p2m, 8 * G->n_p2m);
    if (G->n_p2p) memcpy(p2p, G->p2p, 8 * G->n_p2p);
}

/* Field of one node at x_i (per unit G): monopole (+ quadrupole). */
static void p2m_term(const onode *nd, const double *com, double M, const double *Q, const double *x, int quad,
                     double a[3], double *p)
{
    double d0 = com[0] - x[0], d1 = com[1] - x[1], d2 = com[2] - x[2];
    double r2 = d0 * d0 + d1 * d1 + d2 * d2;
    double r = sqrt(r2);
    double ir = 1.0 / r, ir3 = ir * ir * ir;
    a[0] = M * d0 * ir3;
    a[1] = M * d1 * ir3;
    a[2] = M * d2 * ir3;
    *p = -M * ir;
    (void)nd;
    if (quad) {
        double ir5 = ir3 * ir * ir, ir7 = ir5 * ir * ir;
        double Qd0 = Q[0] * d0 + Q[3] * d1 + Q[4] * d2;
        double Qd1 = Q[3] * d0 + Q[1] * d1 + Q[5] * d2;
        double Qd2 = Q[4] * d0 + Q[5] * d1 + Q[2] * d2;
        double dQd = d0 * Qd0 + d1 * Qd1 + d2 * Qd2;
        a[0] += -Qd0 * ir5 + 2.5 * dQd * d0 * ir7;
        a[1] += -Qd1 * ir5 + 2.5 * dQd * d1 * ir7;
        a[2] += -Qd2 * ir5 + 2.5 * dQd * d2 * ir7;
        *p += -0.5 * dQd * ir5;
    }
}

/* Evaluate the stored lists of target rank r's group, with the given sorted
 * positions/masses and node moments (Mn, comn, Qn arrays of nn entries). */
static void eval_target(const sfgo_tree *t, int64_t r, const double *pos, const double *mass, const double *Mn,
                        const double *comn, const double *Qn, int quad, double a[3], double *phi)
{
    const ogroup *g = &t->groups[t->tgroup[r]];
    double ax = 0, ay = 0, az = 0, p = 0;
    const double *x = pos + 3 * r;
    for (int64_t k = 0; k < g->n_p2m; k++) {
        int64_t ni = g->p2m[k];
        double ta[3], tp;
        p2m_term(&t->nodes[ni], comn + 3 * ni, Mn[ni], Qn + 6 * ni, x, quad, ta, &tp);
        ax += ta[0];
        ay += ta[1];
        az += ta[2];
        p += tp;
    }
    for (int64_t k = 0; k < g->n_p2p; k++) {
        const onode *nd = &t->nodes[g->p2p[k]];
        for (int64_t j = nd->first; j < nd->first + nd->count; j++) {
            if (j == r) continue;
            double dx = pos[3 * j] - x[0], dy = pos[3 * j + 1] - x[1], dz = pos[3 * j + 2] - x[2];
            double rr = sqrt(dx * dx + dy * dy + dz * dz);
            double K, P, Kr;
            pair_law(rr, t->soft[r], t->soft[j], t->sink[r], t->sink[j], &K, &P, &Kr);
            ax += mass[j] * K * dx;
            ay += mass[j] * K * dy;
            az += mass[j] * K * dz;
            p += mass[j] * P;
        }
    }
    a[0] = ax;
    a[1] = ay;
    a[2] = az;
    *phi = p;
}

static void gather_moments(const sfgo_tree *t, double *Mn, double *comn, double *Qn)
{
    for (int64_t i = 0; i < t->nn; i++) {
        Mn[i] = t->nodes[i].M;
        for (int a = 0; a < 3; a++) comn[3 * i + a] = t->nodes[i].com[a];
        for (int c = 0; c < 6; c++) Qn[6 * i + c] = t->nodes[i].Q[c];
    }
}

/* Group-form tree field at the listed original indices (each must be in the
 * active set of the last walk and its group walked).  Returns -1 on a bad row. */
int sfgo_accel_group(const sfgo_tree *t, double G, int quad, const int64_t *idx, int64_t n_idx, double *acc,
                     double *phi)
{
    double *Mn = (double *)malloc(8 * t->nn), *comn = (double *)malloc(24 * t->nn), *Qn = (double *)malloc(48 * t->nn);
    gather_moments(t, Mn, comn, Qn);
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < n_idx; k++) {
        int64_t r = t->rank[idx[k]];
        if (t->tgroup[r] < 0 || !t->groups[t->tgroup[r]].walked) {
            bad = 1;
            continue;
        }
        double a[3], p;
        eval_target(t, r, t->pos, t->mass, Mn, comn, Qn, quad, a, &p);
        for (int c = 0; c < 3; c++) acc[3 * k + c] = G * a[c];
        phi[k] = G * p;
    }
    free(Mn); free(comn); free(Qn);
    return bad ? -1 : 0;
}

/* Tidal term of one node at x_i (per unit G): the derivative -d a / d d of its
 * monopole (+ quadrupole) field, d = com - x_i, q = d.Qd:
 *   monopole   -M I / r^3 + 3 M d d^T / r^5
 *   quadrupole  Q / r^5 - 5 (Qd d^T + d Qd^T) / r^7 - 5/2 q I / r^7 + 35/2 q d d^T / r^9 */
static void p2m_tidal(const double *com, double M, const double *Q, const double *x, int quad, double T[6])
{
    double d[3] = {com[0] - x[0], com[1] - x[1], com[2] - x[2]};
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double ir = 1.0 / sqrt(r2), ir2 = ir * ir, ir3 = ir2 * ir, ir5 = ir3 * ir2;
    static const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
    for (int c = 0; c < 6; c++) {
        double dd = d[ia[c]] * d[ib[c]];
        T[c] += 3.0 * M * dd * ir5 - (c < 3 ? M * ir3 : 0.0);
    }
    if (quad) {
        double ir7 = ir5 * ir2, ir9 = ir7 * ir2;
        double Qd[3] = {Q[0] * d[0] + Q[3] * d[1] + Q[4] * d[2], Q[3] * d[0] + Q[1] * d[1] + Q[5] * d[2],
                        Q[4] * d[0] + Q[5] * d[1] + Q[2] * d[2]};
        double q = d[0] * Qd[0] + d[1] * Qd[1] + d[2] * Qd[2];
        for (int c = 0; c < 6; c++) {
            int a = ia[c], b = ib[c];
            T[c] += Q[c] * ir5 - 5.0 * (Qd[a] * d[b] + d[a] * Qd[b]) * ir7 + 17.5 * q * d[a] * d[b] * ir9 -
                    (c < 3 ? 2.5 * q * ir7 : 0.0);
        }
    }
}

/* Group-form tidal tensor at the listed original indices: the same lists as
 * sfgo_accel_group, with pair and node terms differentiated once more
 * (Sec. 2.2: T in the same pass and with the same opening criterion as g). */
int sfgo_tidal_group(const sfgo_tree *t, double G, int quad, const int64_t *idx, int64_t n_idx, double *tidal)
{
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < n_idx; k++) {
        int64_t r = t->rank[idx[k]];
        if (t->tgroup[r] < 0 || !t->groups[t->tgroup[r]].walked) {
            bad = 1;
            continue;
        }
        const ogroup *g = &t->groups[t->tgroup[r]];
        const double *x = t->pos + 3 * r;
        double T[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t q = 0; q < g->n_p2m; q++) {
            const onode *nd = &t->nodes[g->p2m[q]];
            p2m_tidal(nd->com, nd->M, nd->Q, x, quad, T);
        }
        for (int64_t q = 0; q < g->n_p2p; q++) {
            const onode *nd = &t->nodes[g->p2p[q]];
            for (int64_t j = nd->first; j < nd->first + nd->count; j++) {
                if (j == r) continue;
                double dx = t->pos[3 * j] - x[0], dy = t->pos[3 * j + 1] - x[1], dz = t->pos[3 * j + 2] - x[2];
                double rr = sqrt(dx * dx + dy * dy + dz * dz);
                double K, P, Kr;
                pair_law(rr, t->soft[r], t->soft[j], t->sink[r], t->sink[j], &K, &P, &Kr);
                pair_tidal(t->mass[j], K, Kr, dx, dy, dz, T);
            }
        }
        for (int c = 0; c < 6; c++) tidal[6 * k + c] = G * T[c];
    }
    return bad ? -1 : 0;
}

/* Group-form jerk at the listed original indices on the last walk's lists,
 * vel [n][3] in the input order.  Pairs as sfgo_direct_jerk; an accepted node
 * contributes its monopole term (Sec. 2.2 sums T and j from the monopole
 * contributions of nodes): M [w / r^3 - 3 (d . w) d / r^5], d = com - x_i,
 * w = v_com - v_i, with the node's mass-weighted velocity v_com summed like
 * the centre of mass (members in sorted order, children in octant order). */
int sfgo_jerk_group(const sfgo_tree *t, const double *vel, double G, const int64_t *idx, int64_t n_idx,
                    double *jerk)
{
    int64_t n = t->n, nn = t->nn;
    double *vs = (double *)malloc(24 * n), *pn = (double *)malloc(24 * nn), *vn = (double *)malloc(24 * nn);
    for (int64_t r = 0; r < n; r++)
        for (int a = 0; a < 3; a++) vs[3 * r + a] = vel[3 * t->order[r] + a];
    for (int64_t i = nn - 1; i >= 0; i--) { /* node momenta, then velocities */
        const onode *nd = &t->nodes[i];
        double p[3] = {0, 0, 0};
        if (nd->nchild == 0) {
            for (int64_t k = nd->first; k < nd->first + nd->count; k++)
                for (int a = 0; a < 3; a++) p[a] = p[a] + t->mass[k] * vs[3 * k + a];
        } else {
            for (int q = 0; q < nd->nchild; q++)
                for (int a = 0; a < 3; a++) p[a] = p[a] + pn[3 * (nd->child_first + q) + a];
        }
        for (int a = 0; a < 3; a++) {
            pn[3 * i + a] = p[a];
            vn[3 * i + a] = nd->M > 0.0 ? p[a] / nd->M : 0.0;
        }
    }
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < n_idx; k++) {
        int64_t r = t->rank[idx[k]];
        if (t->tgroup[r] < 0 || !t->groups[t->tgroup[r]].walked) {
            bad = 1;
            continue;
        }
        const ogroup *g = &t->groups[t->tgroup[r]];
        const double *x = t->pos + 3 * r, *v = vs + 3 * r;
        double J[3] = {0, 0, 0};
        for (int64_t q = 0; q < g->n_p2m; q++) {
            int64_t ni = g->p2m[q];
            const onode *nd = &t->nodes[ni];
            double d[3], w[3];
            for (int a = 0; a < 3; a++) {
                d[a] = nd->com[a] - x[a];
                w[a] = vn[3 * ni + a] - v[a];
            }
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double ir = 1.0 / sqrt(r2), ir3 = ir * ir * ir;
            pair_jerk(nd->M, ir3, -3.0 * ir3 * ir * ir, d, w, J);
        }
        for (int64_t q = 0; q < g->n_p2p; q++) {
            const onode *nd = &t->nodes[g->p2p[q]];
            for (int64_t j = nd->first; j < nd->first + nd->count; j++) {
                if (j == r) continue;
                double d[3], w[3];
                for (int a = 0; a < 3; a++) {
                    d[a] = t->pos[3 * j + a] - x[a];
                    w[a] = vs[3 * j + a] - v[a];
                }
                double rr = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                double K, P, Kr;
                pair_law(rr, t->soft[r], t->soft[j], t->sink[r], t->sink[j], &K, &P, &Kr);
                pair_jerk(t->mass[j], K, Kr, d, w, J);
            }
        }
        for (int a = 0; a < 3; a++) jerk[3 * k + a] = G * J[a];
    }
    free(vs); free(pn); free(vn);
    return bad ? -1 : 0;
}

/* Sink two-body timestep (Sec. 2.3, Delta t_2-body): per target,
 *   dt = sqrt(eta) / (1 / t_c,min + 1 / t_dyn,min),
 *   t_c = sqrt(r^2 + eps^2) / |v_s' - v_s|,  t_dyn = sqrt((r^2 + eps^2)^{3/2} / (G (m_s + m_s'))),
 * eps the Plummer-equivalent softening h / 2.8.  Over the group's lists (the
 * minima "in the pass through the gravity tree", masses combined within an
 * accepted node): a pair uses eps = max(h_s, h_s') / 2.8, a node its total
 * mass, centre of mass, mass-weighted velocity and eps = h_s / 2.8.  A zero
 * relative velocity gives no crossing-time limit. */
static void tstep_term(double r2, double eps, double dv2, double msum, double G, double *tc, double *td)
{
    double s2 = r2 + eps * eps;
    if (dv2 > 0.0) {
        double t = sqrt(s2 / dv2);
        if (t < *tc) *tc = t;
    }
    double t = sqrt(s2 * sqrt(s2) / (G * msum));
    if (t < *td) *td = t;
}

static double tstep_dt(double tc, double td, double eta)
{
    return sqrt(eta) / (1.0 / tc + 1.0 / td);
}

/* Direct form over all other particles (input order), vel [n][3]. */
void sfgo_direct_tstep(int64_t n, const double *pos, const double *vel, const double *mass, const double *soft,
                       double G, double eta, int64_t nt, const int64_t *targets, double *dt)
{
    for (int64_t t = 0; t < nt; t++) {
        int64_t i = targets[t];
        double tc = HUGE_VAL, td = HUGE_VAL;
        for (int64_t k = 0; k < n; k++) {
            if (k == i) continue;
            double r2 = 0.0, dv2 = 0.0;
            for (int a = 0; a < 3; a++) {
                double d = pos[3 * k + a] - pos[3 * i + a], w = vel[3 * k + a] - vel[3 * i + a];
                r2 += d * d;
                dv2 += w * w;
            }
            double h = soft[i] > soft[k] ? soft[i] : soft[k];
            tstep_term(r2, h / 2.8, dv2, mass[i] + mass[k], G, &tc, &td);
        }
        dt[t] = tstep_dt(tc, td, eta);
    }
}

int sfgo_tstep_group(const sfgo_tree *t, const double *vel, double G, double eta, const int64_t *idx, int64_t n_idx,
                     double *dt)
{
    int64_t n = t->n, nn = t->nn;
    double *vs = (double *)malloc(24 * n), *pn = (double *)malloc(24 * nn), *vn = (double *)malloc(24 * nn);
    for (int64_t r = 0; r < n; r++)
        for (int a = 0; a < 3; a++) vs[3 * r + a] = vel[3 * t->order[r] + a];
    for (int64_t i = nn - 1; i >= 0; i--) {
        const onode *nd = &t->nodes[i];
        double p[3] = {0, 0, 0};
        if (nd->nchild == 0) {
            for (int64_t k = nd->first; k < nd->first + nd->count; k++)
                for (int a = 0; a < 3; a++) p[a] = p[a] + t->mass[k] * vs[3 * k + a];
        } else {
            for (int q = 0; q < nd->nchild; q++)
                for (int a = 0; a < 3; a++) p[a] = p[a] + pn[3 * (nd->child_first + q) + a];
        }
        for (int a = 0; a < 3; a++) {
            pn[3 * i + a] = p[a];
            vn[3 * i + a] = nd->M > 0.0 ? p[a] / nd->M : 0.0;
        }
    }
    int bad = 0;
    for (int64_t k = 0; k < n_idx; k++) {
        int64_t r = t->rank[idx[k]];
        if (t->tgroup[r] < 0 || !t->groups[t->tgroup[r]].walked) {
            bad = 1;
            continue;
        }
        const ogroup *g = &t->groups[t->tgroup[r]];
        const double *x = t->pos + 3 * r, *v = vs + 3 * r;
        double tc = HUGE_VAL, td = HUGE_VAL;
        for (int64_t q = 0; q < g->n_p2m; q++) {
            int64_t ni = g->p2m[q];
            const onode *nd = &t->nodes[ni];
            double r2 = 0.0, dv2 = 0.0;
            for (int a = 0; a < 3; a++) {
                double d = nd->com[a] - x[a], w = vn[3 * ni + a] - v[a];
                r2 += d * d;
                dv2 += w * w;
            }
            tstep_term(r2, t->soft[r] / 2.8, dv2, t->mass[r] + nd->M, G, &tc, &td);
        }
        for (int64_t q = 0; q < g->n_p2p; q++) {
            const onode *nd = &t->nodes[g->p2p[q]];
            for (int64_t j = nd->first; j < nd->first + nd->count; j++) {
                if (j == r) continue;
                double r2 = 0.0, dv2 = 0.0;
                for (int a = 0; a < 3; a++) {
                    double d = t->pos[3 * j + a] - x[a], w = vs[3 * j + a] - v[a];
                    r2 += d * d;
                    dv2 += w * w;
                }
                double h = t->soft[r] > t->soft[j] ? t->soft[r] : t->soft[j];
                tstep_term(r2, h / 2.8, dv2, t->mass[r] + t->mass[j], G, &tc, &td);
            }
        }
        dt[k] = tstep_dt(tc, td, eta);
    }
    free(vs); free(pn); free(vn);
    return bad ? -1 : 0;
}

/* Frozen-list re-evaluation with new positions/masses (original order):
 * the topology and the lists of the last walk are kept; the moments are
 * recomputed by the same hierarchical combination. */
int sfgo_eval_frozen(const sfgo_tree *t0, double G, int quad, const double *pos, const double *mass,
                     const int64_t *idx, int64_t n_idx, double *acc, double *phi)
{
    sfgo_tree t = *t0;
    int64_t n = t0->n;
    double *spos = (double *)malloc(24 * n), *smass = (double *)malloc(8 * n);
    for (int64_t r = 0; r < n; r++) {
        int64_t i = t0->order[r];
        for (int a = 0; a < 3; a++) spos[3 * r + a] = pos[3 * i + a];
        smass[r] = mass[i];
    }
    t.nodes = (onode *)malloc(sizeof(onode) * t0->nn);
    memcpy(t.nodes, t0->nodes, sizeof(onode) * t0->nn);
    compute_moments(&t, spos, smass);
    double *Mn = (double *)malloc(8 * t.nn), *comn = (double *)malloc(24 * t.nn), *Qn = (double *)malloc(48 * t.nn);
    gather_moments(&t, Mn, comn, Qn);
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < n_idx; k++) {
        int64_t r = t.rank[idx[k]];
        if (t.tgroup[r] < 0 || !t.groups[t.tgroup[r]].walked) {
            bad = 1;
            continue;
        }
        double a[3], p;
        eval_target(&t, r, spos, smass, Mn, comn, Qn, quad, a, &p);
        for (int c = 0; c < 3; c++) acc[3 * k + c] = G * a[c];
        phi[k] = G * p;
    }
    free(Mn); free(comn); free(Qn); free(spos); free(smass); free(t.nodes);
    return bad ? -1 : 0;
}

/* ---------------- per-particle, paper-faithful FP64 opening rule --------- */
static int accept_pp(const sfgo_tree *t, const onode *nd, const double *x, double h, double theta, double gp)
{
    double L = ldexp(t->L0, -nd->level);
    double d0 = nd->com[0] - x[0], d1 = nd->com[1] - x[1], d2 = nd->com[2] - x[2];
    double r2 = d0 * d0 + d1 * d1 + d2 * d2;
    if (!(L * L <= theta * theta * r2)) return 0;
    double b2 = 0.0;
    for (int a = 0; a < 3; a++) {
        double g = 0.0;
        if (nd->flo[a] - x[a] > g) g = nd->flo[a] - x[a];
        if (x[a] - nd->fhi[a] > g) g = x[a] - nd->fhi[a];
        b2 += g * g;
    }
    double hh = h > nd->hmax ? h : nd->hmax;
    if (!(b2 >= hh * hh)) return 0;
    if (gp < 0.0) return 1;
    /* relative criterion, per target: G M L^2 <= alpha |g_prev| r^4 */
    return t->Grel * nd->M * L * L <= t->alpha * gp * r2 * r2;
}

static void walk_pp(const sfgo_tree *t, int64_t r, int64_t ni, double theta, int quad, double a[3], double *p,
                    int64_t *cnt)
{
    const onode *nd = &t->nodes[ni];
    const double *x = t->pos + 3 * r;
    if (accept_pp(t, nd, x, t->soft[r], theta, t->gprev ? t->gprev[r] : -1.0)) {
        double ta[3], tp;
        p2m_term(nd, nd->com, nd->M, nd->Q, x, quad, ta, &tp);
        for (int c = 0; c < 3; c++) a[c] += ta[c];
        *p += tp;
        cnt[1]++;
    } else if (nd->nchild == 0) {
        for (int64_t j = nd->first; j < nd->first + nd->count; j++) {
            if (j == r) continue;
            double dx = t->pos[3 * j] - x[0], dy = t->pos[3 * j + 1] - x[1], dz = t->pos[3 * j + 2] - x[2];
            double rr = sqrt(dx * dx + dy * dy + dz * dz);
            double K, P, Kr;
            pair_law(rr, t->soft[r], t->soft[j], t->sink[r], t->sink[j], &K, &P, &Kr);
            a[0] += t->mass[j] * K * dx;
            a[1] += t->mass[j] * K * dy;
            a[2] += t->mass[j] * K * dz;
            *p += t->mass[j] * P;
            cnt[0]++;
        }
    } else {
        for (int c = 0; c < nd->nchild; c++) walk_pp(t, r, nd->child_first + c, theta, quad, a, p, cnt);
    }
}

/* Per-particle tree field at original indices idx; counts[2*k] = P2P pairs,
 * counts[2*k+1] = P2M nodes. */
void sfgo_accel_pp(const sfgo_tree *t, double G, double theta, int quad, const int64_t *idx, int64_t n_idx,
                   double *acc, double *phi, int64_t *counts)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < n_idx; k++) {
        int64_t r = t->rank[idx[k]];
        double a[3] = {0, 0, 0}, p = 0;
        int64_t cnt[2] = {0, 0};
        walk_pp(t, r, 0, theta, quad, a, &p, cnt);
        for (int c = 0; c < 3; c++) acc[3 * k + c] = G * a[c];
        phi[k] = G * p;
        if (counts) {
            counts[2 * k] = cnt[0];
            counts[2 * k + 1] = cnt[1];
        }
    }
}

/* ---------------- adjoint (VJP) of the group form, lists frozen ---------- */
/* L = sum_rows cot_a . a + cot_phi * phi.  Outputs d_pos[n][3], d_mass[n] in
 * original order (overwritten).  Every group holding a row must be walked. */
int sfgo_vjp(const sfgo_tree *t, double G, int quad, const int64_t *rows, int64_t n_rows, const double *cot_a,
             const double *cot_phi, double *d_pos, double *d_mass)
{
    int64_t n = t->n, nn = t->nn;
    double *ca = (double *)calloc(3 * n, 8), *cp = (double *)calloc(n, 8);
    uint8_t *has = (uint8_t *)calloc(n, 1);
    for (int64_t k = 0; k < n_rows; k++) {
        int64_t r = t->rank[rows[k]];
        if (t->tgroup[r] < 0 || !t->groups[t->tgroup[r]].walked) {
            free(ca); free(cp); free(has);
            return -1;
        }
        for (int c = 0; c < 3; c++) ca[3 * r + c] += cot_a[3 * k + c];
        cp[r] += cot_phi[k];
        has[r] = 1;
    }
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    /* per-thread accumulators: particle grads (sorted order) and node grads */
    double *gp = (double *)calloc((size_t)nthr * 4 * n, 8);
    double *gn = (double *)calloc((size_t)nthr * 10 * nn, 8); /* gM, gcom[3], gQ sym[6] */
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *P = gp + (size_t)tid * 4 * n;
        double *N = gn + (size_t)tid * 10 * nn;
#pragma omp for schedule(dynamic, 64)
        for (int64_t r = 0; r < n; r++) {
            if (!has[r]) continue;
            const ogroup *g = &t->groups[t->tgroup[r]];
            const double *x = t->pos + 3 * r;
            double c0 = ca[3 * r], c1 = ca[3 * r + 1], c2 = ca[3 * r + 2], cf = cp[r];
            for (int64_t k = 0; k < g->n_p2m; k++) {
                int64_t ni = g->p2m[k];
                const onode *nd = &t->nodes[ni];
                const double *Q = nd->Q;
                double M = nd->M;
                double d0 = nd->com[0] - x[0], d1 = nd->com[1] - x[1], d2 = nd->com[2] - x[2];
                double r2 = d0 * d0 + d1 * d1 + d2 * d2, rr = sqrt(r2);
                double ir = 1.0 / rr, ir3 = ir * ir * ir, ir5 = ir3 * ir * ir, ir7 = ir5 * ir * ir, ir9 = ir7 * ir * ir;
                double cd = c0 * d0 + c1 * d1 + c2 * d2;
                /* monopole: a = M d ir3, phi = -M ir */
                double gd0 = M * (c0 * ir3 - 3.0 * cd * d0 * ir5) + cf * M * d0 * ir3;
                double gd1 = M * (c1 * ir3 - 3.0 * cd * d1 * ir5) + cf * M * d1 * ir3;
                double gd2 = M * (c2 * ir3 - 3.0 * cd * d2 * ir5) + cf * M * d2 * ir3;
                double gM = cd * ir3 - cf * ir;
                double gS[6] = {0, 0, 0, 0, 0, 0};
                if (quad) {
                    double Qd0 = Q[0] * d0 + Q[3] * d1 + Q[4] * d2;
                    double Qd1 = Q[3] * d0 + Q[1] * d1 + Q[5] * d2;
                    double Qd2 = Q[4] * d0 + Q[5] * d1 + Q[2] * d2;
                    double Qc0 = Q[0] * c0 + Q[3] * c1 + Q[4] * c2;
                    double Qc1 = Q[3] * c0 + Q[1] * c1 + Q[5] * c2;
                    double Qc2 = Q[4] * c0 + Q[5] * c1 + Q[2] * c2;
                    double dQd = d0 * Qd0 + d1 * Qd1 + d2 * Qd2;
                    double cQd = c0 * Qd0 + c1 * Qd1 + c2 * Qd2;
                    /* c . (-Q d ir5) */
                    gd0 += -Qc0 * ir5 + 5.0 * cQd * d0 * ir7;
                    gd1 += -Qc1 * ir5 + 5.0 * cQd * d1 * ir7;
                    gd2 += -Qc2 * ir5 + 5.0 * cQd * d2 * ir7;
                    /* c . (2.5 dQd d ir7) */
                    gd0 += 2.5 * (2.0 * cd * Qd0 * ir7 + dQd * c0 * ir7 - 7.0 * dQd * cd * d0 * ir9);
                    gd1 += 2.5 * (2.0 * cd * Qd1 * ir7 + dQd * c1 * ir7 - 7.0 * dQd * cd * d1 * ir9);
                    gd2 += 2.5 * (2.0 * cd * Qd2 * ir7 + dQd * c2 * ir7 - 7.0 * dQd * cd * d2 * ir9);
                    /* cf * (-0.5 dQd ir5) */
                    gd0 += cf * (-Qd0 * ir5 + 2.5 * dQd * d0 * ir7);
                    gd1 += cf * (-Qd1 * ir5 + 2.5 * dQd * d1 * ir7);
                    gd2 += cf * (-Qd2 * ir5 + 2.5 * dQd * d2 * ir7);
                    /* symmetric gradient w.r.t. Q */
                    double s = 2.5 * cd * ir7 - 0.5 * cf * ir5;
                    gS[0] = -c0 * d0 * ir5 + s * d0 * d0;
                    gS[1] = -c1 * d1 * ir5 + s * d1 * d1;
                    gS[2] = -c2 * d2 * ir5 + s * d2 * d2;
                    gS[3] = -0.5 * (c0 * d1 + d0 * c1) * ir5 + s * d0 * d1;
                    gS[4] = -0.5 * (c0 * d2 + d0 * c2) * ir5 + s * d0 * d2;
                    gS[5] = -0.5 * (c1 * d2 + d1 * c2) * ir5 + s * d1 * d2;
                }
                P[4 * r] -= gd0;
                P[4 * r + 1] -= gd1;
                P[4 * r + 2] -= gd2;
                double *nn_ = N + 10 * ni;
                nn_[0] += gM;
                nn_[1] += gd0;
                nn_[2] += gd1;
                nn_[3] += gd2;
                for (int c = 0; c < 6; c++) nn_[4 + c] += gS[c];
            }
            for (int64_t k = 0; k < g->n_p2p; k++) {
                const onode *nd = &t->nodes[g->p2p[k]];
                for (int64_t j = nd->first; j < nd->first + nd->count; j++) {
                    if (j == r) continue;
                    double dx = t->pos[3 * j] - x[0], dy = t->pos[3 * j + 1] - x[1], dz = t->pos[3 * j + 2] - x[2];
                    double rr = sqrt(dx * dx + dy * dy + dz * dz);
                    double K, Pp, Kr;
                    pair_law(rr, t->soft[r], t->soft[j], t->sink[r], t->sink[j], &K, &Pp, &Kr);
                    double m = t->mass[j];
                    double cd = c0 * dx + c1 * dy + c2 * dz;
                    double l0 = m * (K * c0 + Kr * cd * dx + cf * K * dx);
                    double l1 = m * (K * c1 + Kr * cd * dy + cf * K * dy);
                    double l2 = m * (K * c2 + Kr * cd * dz + cf * K * dz);
                    P[4 * j] += l0;
                    P[4 * j + 1] += l1;
                    P[4 * j + 2] += l2;
                    P[4 * r] -= l0;
                    P[4 * r + 1] -= l1;
                    P[4 * r + 2] -= l2;
                    P[4 * j + 3] += K * cd + Pp * cf;
                }
            }
        }
    }
    /* reduce thread accumulators in thread order */
    for (int th = 1; th < nthr; th++) {
        for (int64_t k = 0; k < 4 * n; k++) gp[k] += gp[(size_t)th * 4 * n + k];
        for (int64_t k = 0; k < 10 * nn; k++) gn[k] += gn[(size_t)th * 10 * nn + k];
    }
    /* node gradients to member particles: for every ancestor of k,
     * M = sum m, com = sum m x / M, Q = sum m (3 s s^T - s^2 I), s = x - com. */
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n; r++) {
        /* find the leaf of r: deepest node containing r */
        int64_t ni = 0;
        while (t->nodes[ni].nchild != 0) {
            const onode *nd = &t->nodes[ni];
            int64_t next = -1;
            for (int c = 0; c < nd->nchild; c++) {
                const onode *ch = &t->nodes[nd->child_first + c];
                if (r >= ch->first && r < ch->first + ch->count) {
                    next = nd->child_first + c;
                    break;
                }
            }
            ni = next;
        }
        double m = t->mass[r];
        const double *x = t->pos + 3 * r;
        for (; ni >= 0; ni = t->nodes[ni].parent) {
            const onode *nd = &t->nodes[ni];
            const double *g = gn + 10 * ni;
            gp[4 * r + 3] += g[0];
            if (!(nd->M > 0.0)) continue;
            double s0 = x[0] - nd->com[0], s1 = x[1] - nd->com[1], s2 = x[2] - nd->com[2];
            double ss = s0 * s0 + s1 * s1 + s2 * s2;
            const double *S = g + 4;
            double tr = S[0] + S[1] + S[2];
            double Ss0 = S[0] * s0 + S[3] * s1 + S[4] * s2;
            double Ss1 = S[3] * s0 + S[1] * s1 + S[5] * s2;
            double Ss2 = S[4] * s0 + S[5] * s1 + S[2] * s2;
            double sSs = s0 * Ss0 + s1 * Ss1 + s2 * Ss2;
            gp[4 * r + 3] += (g[1] * s0 + g[2] * s1 + g[3] * s2) / nd->M + 3.0 * sSs - ss * tr;
            gp[4 * r] += m / nd->M * g[1] + m * (6.0 * Ss0 - 2.0 * tr * s0);
            gp[4 * r + 1] += m / nd->M * g[2] + m * (6.0 * Ss1 - 2.0 * tr * s1);
            gp[4 * r + 2] += m / nd->M * g[3] + m * (6.0 * Ss2 - 2.0 * tr * s2);
        }
    }
    for (int64_t r = 0; r < n; r++) {
        int64_t i = t->order[r];
        for (int c = 0; c < 3; c++) d_pos[3 * i + c] = G * gp[4 * r + c];
        d_mass[i] = G * gp[4 * r + 3];
    }
    free(ca); free(cp); free(has); free(gp); free(gn);
    return 0;
}

int sfgo_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
