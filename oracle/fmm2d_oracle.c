/*
 * Plain CPU FP64 oracle for the 2D vortex-particle FMM characterised in
 * Cruz & Barba, "Characterization of the errors of the Fast Multipole Method
 * approximation in particle simulations" (2008).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or helper with the CUDA path.
 *
 * Everything is FP64 (double, double complex), in the paper's notation:
 *   z = x + j y,  c_i = -j Gamma_i / (2 pi)          (Sec. 3.2.1, Eq. 20)
 *   ME  a_m = sum_i c_i (z_i - z_*)^m,  m = 0..p-1    (Eqs. 20-21)
 *   M2L L_n += sum_k (-1)^n C(n+k,k) t^-(n+k+1) a_k   (Eq. 22), t = z_b - z_s
 *   M2M b_n  = sum_{k<=n} C(n,k) (z_c - z_P)^(n-k) a_k (Sec. 3.3.2, Eqs. 23-25,
 *              the exact binomial shift; the printed derivation is garbled)
 *   L2L L'_n = sum_{k>=n} C(k,n) (z_c - z_P)^(k-n) L_k (Sec. 3.3.3)
 *   L2P w(y) = sum_n L_n (y - z_b)^n = [u(y)]^*       (Eq. 12 / Sec. 3.2.3)
 *   velocity (u_x, u_y) = (Re w, -Im w)
 *   near field: regularised kernel K_sigma (Eq. 6) over the local list, i != j
 *   (Eq. 9, Eq. 10).
 *   cutoff a (Sec. 4.1, Eq. 29): a pair closer than a keeps K_sigma even when
 *   its leaves are not neighbours; a = 0 is the plain 3x3 rule.
 *
 * Parity status of each function is stated beside it; the pins live in the
 * test suite.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_INVALID_ARG 1
#define ORC_OUT_OF_DOMAIN 2
#define ORC_NONFINITE 3

static const double ORC_PI = 3.14159265358979323846264338327950288;

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Quadtree (Sec. 3.3, Fig. 6): uniform levels, 4^l boxes at level l.        */
/* ------------------------------------------------------------------------ */

/* Leaf coordinates of one point.  The leaf index along an axis is
 * floor((x - x0) * (2^L / W)) in FP64, clamped into [0, 2^L - 1] so that the
 * upper edge of the root box belongs to the last leaf.  A point outside the
 * closed root box is an error.  (The paper is silent on the root box and on
 * points lying on box edges; this is the adopted reading.) */
static int leaf_coord(double x, double x0, double W, int L, uint32_t* out) {
    if (!isfinite(x)) return ORC_NONFINITE;
    if (x < x0 || x > x0 + W) return ORC_OUT_OF_DOMAIN;
    double scale = ldexp(1.0, L) / W;
    double f = floor((x - x0) * scale);
    double top = ldexp(1.0, L) - 1.0;
    if (f > top) f = top;
    if (f < 0.0) f = 0.0;
    *out = (uint32_t)f;
    return ORC_OK;
}

/* Bit-interleaved (Morton) key: leaf x index in the even bits, y in the odd. */
static uint32_t interleave(uint32_t ix, uint32_t iy, int L) {
    uint32_t k = 0;
    for (int b = 0; b < L; ++b) {
        k |= ((ix >> b) & 1u) << (2 * b);
        k |= ((iy >> b) & 1u) << (2 * b + 1);
    }
    return k;
}

static void deinterleave(uint32_t k, int L, uint32_t* ix, uint32_t* iy) {
    uint32_t a = 0, b = 0;
    for (int i = 0; i < L; ++i) {
        a |= ((k >> (2 * i)) & 1u) << i;
        b |= ((k >> (2 * i + 1)) & 1u) << i;
    }
    *ix = a;
    *iy = b;
}

int orc_morton_keys(int64_t n, const double* x, const double* y, double x0, double y0,
                    double W, int L, uint32_t* key) {
    if (n < 0 || L < 0 || L > 15 || !(W > 0.0)) return ORC_INVALID_ARG;
    for (int64_t i = 0; i < n; ++i) {
        uint32_t ix, iy;
        int s = leaf_coord(x[i], x0, W, L, &ix);
        if (s) return s;
        s = leaf_coord(y[i], y0, W, L, &iy);
        if (s) return s;
        key[i] = interleave(ix, iy, L);
    }
    return ORC_OK;
}

/* Stable counting sort by key: particles with equal keys keep input order.
 * perm[r] = input index of the r-th sorted particle; leaf_start has 4^L + 1
 * entries and leaf k holds sorted positions [leaf_start[k], leaf_start[k+1]). */
void orc_sort_by_key(int64_t n, const uint32_t* key, int L, uint32_t* perm,
                     uint32_t* leaf_start) {
    int64_t nleaf = (int64_t)1 << (2 * L);
    uint32_t* count = (uint32_t*)calloc((size_t)nleaf + 1, sizeof(uint32_t));
    for (int64_t i = 0; i < n; ++i) count[key[i] + 1] += 1;
    for (int64_t k = 0; k < nleaf; ++k) count[k + 1] += count[k];
    memcpy(leaf_start, count, ((size_t)nleaf + 1) * sizeof(uint32_t));
    for (int64_t i = 0; i < n; ++i) perm[count[key[i]]++] = (uint32_t)i;
    free(count);
}

/* ------------------------------------------------------------------------ */
/* Kernels (Sec. 2, Eq. 6; Sec. 4.1, Eqs. 26-27).                             */
/* ------------------------------------------------------------------------ */

/* Regularised Biot-Savart kernel of Eq. 6 at separation (dx, dy), times
 * Gamma.  K_sigma(0) = 0 by its limit, so a zero separation contributes
 * nothing.  1 - exp(-q) is formed as -expm1(-q) to keep it accurate for small
 * q. */
static void k_sigma(double dx, double dy, double gamma, double sigma, double* u, double* v) {
    double r2 = dx * dx + dy * dy;
    if (r2 == 0.0) return;
    double f = gamma * (-expm1(-r2 / (2.0 * sigma * sigma))) / (2.0 * ORC_PI * r2);
    *u += -dy * f;
    *v += dx * f;
}

/* Singular kernel K' of Eq. 27 (equivalently Eq. 15): (-y, x) / (2 pi r^2). */
static void k_singular(double dx, double dy, double gamma, double* u, double* v) {
    double r2 = dx * dx + dy * dy;
    if (r2 == 0.0) return;
    double f = gamma / (2.0 * ORC_PI * r2);
    *u += -dy * f;
    *v += dx * f;
}

/* O1: discrete Biot-Savart sum of Eq. 7 evaluated at source points, with the
 * self term excluded as in Eq. 9.  targets[t] are particle indices; the
 * velocity at each is written to (u[t], v[t]). */
int orc_direct(int64_t n, const double* x, const double* y, const double* gamma, double sigma,
               int64_t ntarg, const int64_t* targets, double* u, double* v) {
    if (n < 0 || ntarg < 0 || !(sigma > 0.0)) return ORC_INVALID_ARG;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < ntarg; ++t) {
        int64_t i = targets[t];
        double su = 0.0, sv = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            k_sigma(x[i] - x[j], y[i] - y[j], gamma[j], sigma, &su, &sv);
        }
        u[t] = su;
        v[t] = sv;
    }
    return ORC_OK;
}

/* O2: the sum the FMM converges to as p grows.  Pairs whose leaves are in
 * each other's local list (the 3x3 leaf neighbourhood, Sec. 3.3.1) use the
 * regularised kernel, and so does every pair closer than the cutoff a
 * (Sec. 4.1: below the distance a the regularised kernel is kept); every
 * other pair uses the singular kernel, as the far field does (Eq. 10,
 * Sec. 4.1).  a = 0 gives the plain 3x3 rule. */
int orc_hybrid_cut(int64_t n, const double* x, const double* y, const double* gamma,
                   double sigma, double x0, double y0, double W, int L, double a, int64_t ntarg,
                   const int64_t* targets, double* u, double* v) {
    if (n < 0 || ntarg < 0 || !(sigma > 0.0) || !(W > 0.0) || L < 0 || L > 15 || !(a >= 0.0))
        return ORC_INVALID_ARG;
    uint32_t* lx = (uint32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(uint32_t));
    uint32_t* ly = (uint32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(uint32_t));
    int status = ORC_OK;
    for (int64_t i = 0; i < n && status == ORC_OK; ++i) {
        status = leaf_coord(x[i], x0, W, L, &lx[i]);
        if (status == ORC_OK) status = leaf_coord(y[i], y0, W, L, &ly[i]);
    }
    if (status == ORC_OK) {
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t t = 0; t < ntarg; ++t) {
            int64_t i = targets[t];
            double su = 0.0, sv = 0.0;
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                int64_t ddx = (int64_t)lx[i] - (int64_t)lx[j];
                int64_t ddy = (int64_t)ly[i] - (int64_t)ly[j];
                double dx = x[i] - x[j], dy = y[i] - y[j];
                int near = (ddx >= -1 && ddx <= 1 && ddy >= -1 && ddy <= 1) ||
                           dx * dx + dy * dy < a * a;
                if (near)
                    k_sigma(dx, dy, gamma[j], sigma, &su, &sv);
                else
                    k_singular(dx, dy, gamma[j], &su, &sv);
            }
            u[t] = su;
            v[t] = sv;
        }
    }
    free(lx);
    free(ly);
    return status;
}

int orc_hybrid(int64_t n, const double* x, const double* y, const double* gamma, double sigma,
               double x0, double y0, double W, int L, int64_t ntarg, const int64_t* targets,
               double* u, double* v) {
    return orc_hybrid_cut(n, x, y, gamma, sigma, x0, y0, W, L, 0.0, ntarg, targets, u, v);
}

/* ------------------------------------------------------------------------ */
/* Expansions and translation operators (Sec. 3.2 - 3.3).  Coefficient arrays */
/* are p complex numbers stored as interleaved (re, im) doubles.              */
/* ------------------------------------------------------------------------ */

/* Binomial coefficient C(n, k) from Pascal's triangle (exact in FP64 for the
 * sizes used here, n <= 2p <= 128 gives values far beyond 2^53 only for
 * p > 28; those are still correctly rounded sums of exact integers). */
static double* binomial_table(int nmax) {
    double* c = (double*)calloc((size_t)(nmax + 1) * (nmax + 1), sizeof(double));
    for (int n = 0; n <= nmax; ++n) {
        c[n * (nmax + 1) + 0] = 1.0;
        for (int k = 1; k <= n; ++k)
            c[n * (nmax + 1) + k] = c[(n - 1) * (nmax + 1) + k - 1] +
                                    (k <= n - 1 ? c[(n - 1) * (nmax + 1) + k] : 0.0);
    }
    return c;
}

/* P2M: a_m = sum_i c_i (z_i - z_*)^m for m = 0..p-1, c_i = -j Gamma_i / 2pi
 * (Eq. 20 truncated as in Eq. 21).  Adds into a. */
static void p2m(int64_t cnt, const int64_t* idx, const double* x, const double* y,
                const double* gamma, double complex zc, int p, double complex* a) {
    for (int64_t q = 0; q < cnt; ++q) {
        int64_t i = idx ? idx[q] : q;
        double complex ci = -I * gamma[i] / (2.0 * ORC_PI);
        double complex d = (x[i] + I * y[i]) - zc;
        double complex pw = 1.0;
        for (int m = 0; m < p; ++m) {
            a[m] += ci * pw;
            pw *= d;
        }
    }
}

/* M2M (Sec. 3.3.2): shift an ME centred at zc to the parent centre zp,
 * b_n += sum_{k=0..n} C(n,k) (zc - zp)^(n-k) a_k.  This is the exact
 * re-expansion of (z_i - zp)^n = ((z_i - zc) + (zc - zp))^n. */
static void m2m(int p, const double* C, int ld, const double complex* a, double complex zc,
                double complex zp, double complex* b) {
    double complex t = zc - zp;
    double complex tp[128];
    tp[0] = 1.0;
    for (int e = 1; e < p; ++e) tp[e] = tp[e - 1] * t;
    for (int n = 0; n < p; ++n) {
        double complex s = 0.0;
        for (int k = 0; k <= n; ++k) s += C[n * ld + k] * tp[n - k] * a[k];
        b[n] += s;
    }
}

/* M2L (Sec. 3.2.3, Eq. 22): L_n += sum_k (-1)^n C(n+k,k) t^-(n+k+1) a_k with
 * t = z_target - z_source (Me_k(y + t) re-expanded in powers of y). */
static void m2l(int p, const double* C, int ld, const double complex* a, double complex zs,
                double complex zt, double complex* Lc) {
    double complex t = zt - zs;
    double complex it = 1.0 / t;
    double complex ip[256];
    ip[0] = 1.0;
    for (int e = 1; e <= 2 * p; ++e) ip[e] = ip[e - 1] * it;
    for (int n = 0; n < p; ++n) {
        double complex s = 0.0;
        for (int k = 0; k < p; ++k) s += C[(n + k) * ld + k] * ip[n + k + 1] * a[k];
        Lc[n] += ((n & 1) ? -1.0 : 1.0) * s;
    }
}

/* L2L (Sec. 3.3.3): L'_n += sum_{k=n..p-1} C(k,n) (zc - zp)^(k-n) L_k, the
 * exact re-expansion of the parent polynomial about the child centre zc. */
static void l2l(int p, const double* C, int ld, const double complex* Lp, double complex zp,
                double complex zc, double complex* Lc) {
    double complex t = zc - zp;
    double complex tp[128];
    tp[0] = 1.0;
    for (int e = 1; e < p; ++e) tp[e] = tp[e - 1] * t;
    for (int n = 0; n < p; ++n) {
        double complex s = 0.0;
        for (int k = n; k < p; ++k) s += C[k * ld + n] * tp[k - n] * Lp[k];
        Lc[n] += s;
    }
}

/* L2P: w(y) = sum_n L_n (y - zc)^n, the conjugate velocity [u(y)]^*. */
static double complex l2p(int p, const double complex* Lc, double complex zc, double complex zy) {
    double complex d = zy - zc, pw = 1.0, w = 0.0;
    for (int n = 0; n < p; ++n) {
        w += Lc[n] * pw;
        pw *= d;
    }
    return w;
}

/* ME evaluated straight at a point: sum_m a_m (y - z_*)^(-m-1) (Eq. 20). */
static double complex me_eval(int p, const double complex* a, double complex zc,
                              double complex zy) {
    double complex id = 1.0 / (zy - zc), pw = id, w = 0.0;
    for (int m = 0; m < p; ++m) {
        w += a[m] * pw;
        pw *= id;
    }
    return w;
}

/* Operator-level entry points, used by the pins on single expansions.
 * Coefficient arrays are interleaved (re, im) doubles of length 2p. */
void orc_op_p2m(int64_t n, const double* x, const double* y, const double* gamma, double cx,
                double cy, int p, double* a_out) {
    memset(a_out, 0, sizeof(double) * 2 * (size_t)p);
    p2m(n, NULL, x, y, gamma, cx + I * cy, p, (double complex*)a_out);
}

void orc_op_m2m(int p, const double* a, double cx, double cy, double px, double py,
                double* b_out) {
    double* C = binomial_table(2 * p);
    memset(b_out, 0, sizeof(double) * 2 * (size_t)p);
    m2m(p, C, 2 * p + 1, (const double complex*)a, cx + I * cy, px + I * py,
        (double complex*)b_out);
    free(C);
}

void orc_op_m2l(int p, const double* a, double sx, double sy, double tx, double ty,
                double* l_out) {
    double* C = binomial_table(2 * p);
    memset(l_out, 0, sizeof(double) * 2 * (size_t)p);
    m2l(p, C, 2 * p + 1, (const double complex*)a, sx + I * sy, tx + I * ty,
        (double complex*)l_out);
    free(C);
}

void orc_op_l2l(int p, const double* l, double px, double py, double cx, double cy,
                double* l_out) {
    double* C = binomial_table(2 * p);
    memset(l_out, 0, sizeof(double) * 2 * (size_t)p);
    l2l(p, C, 2 * p + 1, (const double complex*)l, px + I * py, cx + I * cy,
        (double complex*)l_out);
    free(C);
}

void orc_op_l2p(int p, const double* l, double cx, double cy, int64_t m, const double* yx,
                const double* yy, double* w_out) {
    for (int64_t q = 0; q < m; ++q) {
        double complex w = l2p(p, (const double complex*)l, cx + I * cy, yx[q] + I * yy[q]);
        w_out[2 * q] = creal(w);
        w_out[2 * q + 1] = cimag(w);
    }
}

void orc_op_me_eval(int p, const double* a, double cx, double cy, int64_t m, const double* yx,
                    const double* yy, double* w_out) {
    for (int64_t q = 0; q < m; ++q) {
        double complex w = me_eval(p, (const double complex*)a, cx + I * cy, yx[q] + I * yy[q]);
        w_out[2 * q] = creal(w);
        w_out[2 * q + 1] = cimag(w);
    }
}

/* ------------------------------------------------------------------------ */
/* O3: the plain FMM (Sec. 3.1 call order, Fig. 3).                           */
/*   1. quadtree: leaf of every particle at level L                          */
/*   2. upward sweep: P2M at level L, M2M for levels L-1 .. 2                 */
/*   3. downward sweep: for l = 2 .. L, M2L over the interaction list, and,   */
/*      for l > 2, L2L from the parent                                        */
/*   4. evaluation: L2P + near-field direct sum over the local list           */
/* Levels 0 and 1 carry no expansions; with L < 2 every pair is near field.   */
/* Boxes of level l are indexed row-major, b = iy * 2^l + ix.                 */
/* ------------------------------------------------------------------------ */

static double complex box_centre(double x0, double y0, double W, int l, int64_t ix, int64_t iy) {
    double w = W / ldexp(1.0, l);
    return (x0 + (ix + 0.5) * w) + I * (y0 + (iy + 0.5) * w);
}

/* O3 with the cutoff a of Sec. 4.1: the FMM of Sec. 3.1 (far field through
 * the expansions with the singular kernel, near field over the 3x3 local
 * list with K_sigma), plus, for every pair closer than a whose leaves are not
 * neighbours, the difference K_sigma - K' that turns the singular kernel the
 * far field applied to it back into the regularised one.  a = 0 is the plain
 * FMM. */
int orc_fmm_cut(int64_t n, const double* x, const double* y, const double* gamma, double sigma,
                int p, int L, double x0, double y0, double W, double a, double* u, double* v) {
    if (n < 0 || p < 1 || p > 64 || L < 0 || L > 12 || !(sigma > 0.0) || !(W > 0.0) ||
        !(a >= 0.0) || !isfinite(a))
        return ORC_INVALID_ARG;
    int64_t nl = (int64_t)1 << L; /* leaves per side */
    uint32_t* key = (uint32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(uint32_t));
    int status = orc_morton_keys(n, x, y, x0, y0, W, L, key);
    if (status) {
        free(key);
        return status;
    }
    /* particles of each leaf, leaves indexed row-major */
    uint32_t* rowkey = (uint32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(uint32_t));
    for (int64_t i = 0; i < n; ++i) {
        uint32_t ix, iy;
        deinterleave(key[i], L, &ix, &iy);
        rowkey[i] = (uint32_t)(iy * nl + ix);
    }
    uint32_t* perm = (uint32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(uint32_t));
    uint32_t* start = (uint32_t*)malloc((size_t)(nl * nl + 1) * sizeof(uint32_t));
    orc_sort_by_key(n, rowkey, L, perm, start);
    int64_t* plist = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t r = 0; r < n; ++r) plist[r] = perm[r];

    double* C = binomial_table(2 * p);
    int ld = 2 * p + 1;
    double complex* ME[13] = {0};
    double complex* LE[13] = {0};
    for (int l = 2; l <= L; ++l) {
        int64_t nb = (int64_t)1 << (2 * l);
        ME[l] = (double complex*)calloc((size_t)(nb * p), sizeof(double complex));
        LE[l] = (double complex*)calloc((size_t)(nb * p), sizeof(double complex));
    }

    if (L >= 2) {
        /* upward sweep: P2M at the leaves (Eq. 20) */
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t b = 0; b < nl * nl; ++b) {
            int64_t ix = b % nl, iy = b / nl;
            p2m(start[b + 1] - start[b], plist + start[b], x, y, gamma,
                box_centre(x0, y0, W, L, ix, iy), p, ME[L] + b * p);
        }
        /* M2M for levels L-1 .. 2: each parent gathers its four children */
        for (int l = L - 1; l >= 2; --l) {
            int64_t nb = (int64_t)1 << l;
#pragma omp parallel for schedule(dynamic, 16)
            for (int64_t b = 0; b < nb * nb; ++b) {
                int64_t ix = b % nb, iy = b / nb;
                double complex zp = box_centre(x0, y0, W, l, ix, iy);
                for (int cy = 0; cy < 2; ++cy)
                    for (int cx = 0; cx < 2; ++cx) {
                        int64_t jx = 2 * ix + cx, jy = 2 * iy + cy;
                        m2m(p, C, ld, ME[l + 1] + (jy * 2 * nb + jx) * p,
                            box_centre(x0, y0, W, l + 1, jx, jy), zp, ME[l] + b * p);
                    }
            }
        }
        /* downward sweep */
        for (int l = 2; l <= L; ++l) {
            int64_t nb = (int64_t)1 << l;
#pragma omp parallel for schedule(dynamic, 16)
            for (int64_t b = 0; b < nb * nb; ++b) {
                int64_t ix = b % nb, iy = b / nb;
                double complex zt = box_centre(x0, y0, W, l, ix, iy);
                /* interaction list: children of the parent's neighbours that
                 * are not in this box's local list (Sec. 3.3.1).  Children of
                 * the parent itself are all neighbours of the box, so scanning
                 * the parent's local list gives the same set. */
                int64_t px = ix >> 1, py = iy >> 1;
                for (int64_t qy = py - 1; qy <= py + 1; ++qy)
                    for (int64_t qx = px - 1; qx <= px + 1; ++qx) {
                        if (qx < 0 || qy < 0 || qx >= nb / 2 || qy >= nb / 2) continue;
                        for (int cy = 0; cy < 2; ++cy)
                            for (int cx = 0; cx < 2; ++cx) {
                                int64_t sx = 2 * qx + cx, sy = 2 * qy + cy;
                                if (llabs(sx - ix) <= 1 && llabs(sy - iy) <= 1) continue;
                                m2l(p, C, ld, ME[l] + (sy * nb + sx) * p,
                                    box_centre(x0, y0, W, l, sx, sy), zt, LE[l] + b * p);
                            }
                    }
                /* L2L from the parent, whose LE is complete (level l-1 done) */
                if (l > 2) {
                    l2l(p, C, ld, LE[l - 1] + (py * (nb / 2) + px) * p,
                        box_centre(x0, y0, W, l - 1, px, py), zt, LE[l] + b * p);
                }
            }
        }
    }

    /* evaluation: far field by L2P, near field over the local list */
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t b = 0; b < nl * nl; ++b) {
        int64_t ix = b % nl, iy = b / nl;
        double complex zc = box_centre(x0, y0, W, L, ix, iy);
        for (uint32_t r = start[b]; r < start[b + 1]; ++r) {
            int64_t i = plist[r];
            double su = 0.0, sv = 0.0;
            if (L >= 2) {
                double complex w = l2p(p, LE[L] + b * p, zc, x[i] + I * y[i]);
                su = creal(w);
                sv = -cimag(w);
            }
            for (int64_t qy = iy - 1; qy <= iy + 1; ++qy)
                for (int64_t qx = ix - 1; qx <= ix + 1; ++qx) {
                    if (qx < 0 || qy < 0 || qx >= nl || qy >= nl) continue;
                    int64_t q = qy * nl + qx;
                    for (uint32_t s = start[q]; s < start[q + 1]; ++s) {
                        int64_t j = plist[s];
                        if (j == i) continue;
                        k_sigma(x[i] - x[j], y[i] - y[j], gamma[j], sigma, &su, &sv);
                    }
                }
            /* cutoff: non-neighbour leaves that can hold a source closer than
             * a (leaves at Chebyshev distance d >= 2 are at least (d - 1)
             * leaf widths away) */
            if (a > 0.0) {
                double w = W / ldexp(1.0, L);
                int64_t R = 1 + (int64_t)ceil(a / w);
                for (int64_t qy = iy - R; qy <= iy + R; ++qy)
                    for (int64_t qx = ix - R; qx <= ix + R; ++qx) {
                        if (qx < 0 || qy < 0 || qx >= nl || qy >= nl) continue;
                        if (llabs(qx - ix) <= 1 && llabs(qy - iy) <= 1) continue;
                        int64_t q = qy * nl + qx;
                        for (uint32_t s = start[q]; s < start[q + 1]; ++s) {
                            int64_t j = plist[s];
                            double dx = x[i] - x[j], dy = y[i] - y[j];
                            if (!(dx * dx + dy * dy < a * a)) continue;
                            k_sigma(dx, dy, gamma[j], sigma, &su, &sv);
                            k_singular(dx, dy, -gamma[j], &su, &sv);
                        }
                    }
            }
            u[i] = su;
            v[i] = sv;
        }
    }

    for (int l = 2; l <= L; ++l) {
        free(ME[l]);
        free(LE[l]);
    }
    free(C);
    free(plist);
    free(start);
    free(perm);
    free(rowkey);
    free(key);
    return ORC_OK;
}

int orc_fmm(int64_t n, const double* x, const double* y, const double* gamma, double sigma,
            int p, int L, double x0, double y0, double W, double* u, double* v) {
    return orc_fmm_cut(n, x, y, gamma, sigma, p, L, x0, y0, W, 0.0, u, v);
}

/* ------------------------------------------------------------------------ */
/* Error estimates of Sec. 4.                                                 */
/* ------------------------------------------------------------------------ */

/* Kernel-substitution estimate of Eq. 29, read with the squared distance of
 * Eq. 6 (the printed exponent drops the square):
 *   exp(-a^2 / (2 sigma^2)) * sum_i Gamma_i. */
double orc_kernel_error_estimate(double a, double sigma, double sum_gamma) {
    return exp(-(a * a) / (2.0 * sigma * sigma)) * sum_gamma;
}

/* Truncation bound of Eqs. 30-31, with the garbled last line read as the sum
 * of the geometric tail:  A * b^p / ((1 - b) |y - x_*|), A = |sum Gamma_i| / 2pi. */
double orc_truncation_bound(double A, double b, int p, double dist) {
    return A * pow(b, (double)p) / ((1.0 - b) * dist);
}
