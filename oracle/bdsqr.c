/*
 * oracle/bdsqr.c -- plain, slow FP64 CPU reference for the SVD of an upper
 * bidiagonal matrix.  TEST INFRASTRUCTURE ONLY: nothing on the product path
 * may link, load or call this file; only tests/, the smoke check and the
 * CPU-baseline leg of the benchmark do.
 *
 * What it computes: B = U diag(s) V^T for the n x n upper bidiagonal B with
 * diagonal d[0..n-1] and superdiagonal e[0..n-2], singular values in
 * descending order (the ordering of the paper's problem statement, Sec. 1).
 * The bidiagonal divide-and-conquer of Sec. 4.2 reaches this same SVD up to
 * rounding, so the oracle is that definition computed by the classical
 * method the paper names as the baseline bidiagonal solver (QR iteration,
 * Sec. 2): Golub-Kahan implicit-shift QR sweeps with a Wilkinson shift,
 * chasing a bulge with plane rotations that are accumulated into U and V.
 *
 * Independent checks that do not use QR at all:
 *   oracle_sturm_sigma -- bisection on Sturm counts of the 2n x 2n
 *     Golub-Kahan tridiagonal (zero diagonal, off-diagonal d0,e0,d1,...),
 *     whose eigenvalues are +-s_i.
 *   oracle_residual    -- ||B V - U S||_F / ||B||_F in O(n^2) using the
 *     bidiagonal structure of B.
 *
 * Everything is double precision, single threaded, with no blocking or
 * reordering beyond the textbook sweep.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EPS 2.220446049250313e-16 /* 2^-52 */

/* Plane rotation with c*f + s*g = r, -s*f + c*g = 0. */
static void orc_rot(double f, double g, double *c, double *s, double *r)
{
    if (g == 0.0) { *c = 1.0; *s = 0.0; *r = f; return; }
    if (f == 0.0) { *c = 0.0; *s = 1.0; *r = g; return; }
    double h = hypot(f, g);
    *c = f / h; *s = g / h; *r = h;
}

/* columns a, b of an n-row column-major matrix X:
 * X_a <- c X_a + s X_b ;  X_b <- -s X_a + c X_b */
static void orc_rot_cols(double *X, int n, int ld, int a, int b, double c, double s)
{
    double *xa = X + (size_t)a * ld, *xb = X + (size_t)b * ld;
    for (int i = 0; i < n; ++i) {
        double u = xa[i], v = xb[i];
        xa[i] = c * u + s * v;
        xb[i] = -s * u + c * v;
    }
}

/* One Golub-Kahan implicit-shift QR sweep on the unreduced block [lo, hi]. */
static void orc_gk_sweep(int n, double *d, double *e, int lo, int hi, double *U, double *V)
{
    /* Wilkinson shift: eigenvalue of the trailing 2x2 of B^T B nearer its
     * last diagonal entry. */
    double dm = d[hi - 1], dn = d[hi], em = e[hi - 1];
    double el = (hi - 1 > lo) ? e[hi - 2] : 0.0;
    double t11 = dm * dm + el * el, t22 = dn * dn + em * em, t12 = dm * em;
    double delta = 0.5 * (t11 - t22);
    double sgn = (delta >= 0.0) ? 1.0 : -1.0;
    double denom = delta + sgn * hypot(delta, t12);
    double mu = (denom != 0.0) ? t22 - t12 * t12 / denom : t22;

    double y = d[lo] * d[lo] - mu;
    double z = d[lo] * e[lo];
    for (int k = lo; k < hi; ++k) {
        double c, s, r;
        /* right rotation on columns k, k+1 */
        orc_rot(y, z, &c, &s, &r);
        if (k > lo) e[k - 1] = r;
        double dk = d[k], ek = e[k], dk1 = d[k + 1];
        d[k] = c * dk + s * ek;
        e[k] = -s * dk + c * ek;
        double bulge = s * dk1;
        d[k + 1] = c * dk1;
        if (V) orc_rot_cols(V, n, n, k, k + 1, c, s);
        /* left rotation on rows k, k+1 removes the bulge at (k+1, k) */
        orc_rot(d[k], bulge, &c, &s, &r);
        d[k] = r;
        ek = e[k]; dk1 = d[k + 1];
        e[k] = c * ek + s * dk1;
        d[k + 1] = -s * ek + c * dk1;
        if (k < hi - 1) {
            double ek1 = e[k + 1];
            z = s * ek1;           /* new bulge at (k, k+2) */
            e[k + 1] = c * ek1;
            y = e[k];
        }
        if (U) orc_rot_cols(U, n, n, k, k + 1, c, s);
    }
}

/* d[k] == 0 with k < hi: left rotations with rows k+1..hi clear row k. */
static void orc_chase_row(int n, double *d, double *e, int k, int hi, double *U)
{
    double x = e[k];
    e[k] = 0.0;
    for (int j = k + 1; j <= hi && x != 0.0; ++j) {
        double c, s, r;
        orc_rot(d[j], x, &c, &s, &r);
        d[j] = r;
        if (j < hi) { x = -s * e[j]; e[j] = c * e[j]; }
        if (U) orc_rot_cols(U, n, n, j, k, c, s);
    }
}

/* d[hi] == 0: right rotations with columns hi-1..lo clear column hi. */
static void orc_chase_col(int n, double *d, double *e, int lo, int hi, double *V)
{
    double x = e[hi - 1];
    e[hi - 1] = 0.0;
    for (int j = hi - 1; j >= lo && x != 0.0; --j) {
        double c, s, r;
        orc_rot(d[j], x, &c, &s, &r);
        d[j] = r;
        if (j > lo) { x = -s * e[j - 1]; e[j - 1] = c * e[j - 1]; }
        if (V) orc_rot_cols(V, n, n, j, hi, c, s);
    }
}

/*
 * SVD of the upper bidiagonal (d, e).  s[n] receives the singular values in
 * descending order.  If U and VT are both non-NULL they receive the left
 * vectors (columns of U, column-major, leading dimension ldu) and V^T
 * (column-major, leading dimension ldvt).  Returns 0, or the number of
 * unconverged superdiagonal entries if max_sweeps*n sweeps did not suffice,
 * or -1 on bad arguments / allocation failure.
 */
int oracle_bdsqr(int n, const double *d_in, const double *e_in, double *s,
                 double *U, int ldu, double *VT, int ldvt, int max_sweeps)
{
    if (n < 0 || !s || (n > 0 && !d_in) || (n > 1 && !e_in)) return -1;
    if (n == 0) return 0;
    int want = (U != NULL && VT != NULL);
    if (want && (ldu < n || ldvt < n)) return -1;
    if (max_sweeps <= 0) max_sweeps = 30;

    double *d = (double *)malloc(sizeof(double) * n);
    double *e = (double *)calloc((size_t)n, sizeof(double));
    double *Uw = NULL, *Vw = NULL;
    if (!d || !e) { free(d); free(e); return -1; }
    memcpy(d, d_in, sizeof(double) * n);
    if (n > 1) memcpy(e, e_in, sizeof(double) * (n - 1));
    if (want) {
        Uw = (double *)calloc((size_t)n * n, sizeof(double));
        Vw = (double *)calloc((size_t)n * n, sizeof(double));
        if (!Uw || !Vw) { free(d); free(e); free(Uw); free(Vw); return -1; }
        for (int i = 0; i < n; ++i) { Uw[(size_t)i * n + i] = 1.0; Vw[(size_t)i * n + i] = 1.0; }
    }

    /* The SVD is homogeneous (sigma(cB) = c sigma(B), same vectors): work on
     * B / max|d, e| so that the squares in the shift cannot overflow, and
     * scale the singular values back at the end. */
    double bscale = 0.0;
    for (int i = 0; i < n; ++i) bscale = fmax(bscale, fabs(d[i]));
    for (int i = 0; i + 1 < n; ++i) bscale = fmax(bscale, fabs(e[i]));
    if (bscale > 0.0) {
        for (int i = 0; i < n; ++i) d[i] /= bscale;
        for (int i = 0; i + 1 < n; ++i) e[i] /= bscale;
    }
    double bnorm = 0.0;
    for (int i = 0; i < n; ++i) bnorm = fmax(bnorm, fabs(d[i]));
    for (int i = 0; i + 1 < n; ++i) bnorm = fmax(bnorm, fabs(e[i]));
    double dtiny = ORC_EPS * bnorm;

    long long budget = (long long)max_sweeps * n;
    int info = 0;
    int hi = n - 1;
    while (hi > 0) {
        if (fabs(e[hi - 1]) <= ORC_EPS * (fabs(d[hi - 1]) + fabs(d[hi])) ||
            fabs(e[hi - 1]) <= dtiny * ORC_EPS) {
            e[hi - 1] = 0.0;
            --hi;
            continue;
        }
        int lo = hi - 1;
        while (lo > 0 && fabs(e[lo - 1]) > ORC_EPS * (fabs(d[lo - 1]) + fabs(d[lo])) &&
               fabs(e[lo - 1]) > dtiny * ORC_EPS)
            --lo;
        if (lo > 0) e[lo - 1] = 0.0;
        /* a (numerically) zero diagonal entry splits the block */
        int kz = -1;
        for (int k = lo; k <= hi; ++k)
            if (fabs(d[k]) <= dtiny) { kz = k; break; }
        if (kz >= 0) {
            d[kz] = 0.0;
            if (kz < hi) orc_chase_row(n, d, e, kz, hi, Uw);
            else orc_chase_col(n, d, e, lo, hi, Vw);
            continue;
        }
        if (budget-- <= 0) {
            for (int i = 0; i < hi; ++i) if (e[i] != 0.0) ++info;
            break;
        }
        orc_gk_sweep(n, d, e, lo, hi, Uw, Vw);
    }

    /* non-negative singular values: flip the matching right vector */
    for (int i = 0; i < n; ++i) {
        if (d[i] < 0.0) {
            d[i] = -d[i];
            if (want) for (int r = 0; r < n; ++r) Vw[(size_t)i * n + r] = -Vw[(size_t)i * n + r];
        }
    }
    /* descending order, stable selection (ties keep the lower index first) */
    for (int i = 0; i < n; ++i) {
        int best = i;
        for (int j = i + 1; j < n; ++j) if (d[j] > d[best]) best = j;
        if (best != i) {
            /* rotate [i..best] right by one so equal keys keep their order */
            double t = d[best];
            memmove(d + i + 1, d + i, sizeof(double) * (best - i));
            d[i] = t;
            if (want) {
                double *tmp = (double *)malloc(sizeof(double) * n);
                if (tmp) {
                    memcpy(tmp, Uw + (size_t)best * n, sizeof(double) * n);
                    memmove(Uw + (size_t)(i + 1) * n, Uw + (size_t)i * n, sizeof(double) * n * (best - i));
                    memcpy(Uw + (size_t)i * n, tmp, sizeof(double) * n);
                    memcpy(tmp, Vw + (size_t)best * n, sizeof(double) * n);
                    memmove(Vw + (size_t)(i + 1) * n, Vw + (size_t)i * n, sizeof(double) * n * (best - i));
                    memcpy(Vw + (size_t)i * n, tmp, sizeof(double) * n);
                    free(tmp);
                } else info = -1;
            }
        }
    }
    if (bscale > 0.0)
        for (int i = 0; i < n; ++i) d[i] *= bscale;
    memcpy(s, d, sizeof(double) * n);
    if (want) {
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) U[(size_t)j * ldu + i] = Uw[(size_t)j * n + i];
        for (int i = 0; i < n; ++i)          /* VT row i = V column i */
            for (int j = 0; j < n; ++j) VT[(size_t)j * ldvt + i] = Vw[(size_t)i * n + j];
    }
    free(d); free(e); free(Uw); free(Vw);
    return info;
}

/*
 * Number of eigenvalues smaller than x of the 2n x 2n Golub-Kahan
 * tridiagonal T with zero diagonal and off-diagonal (d0, e0, d1, e1, ...,
 * e_{n-2}, d_{n-1}), by the signs of the LDL^T pivots of T - x I.
 */
long oracle_sturm_count(int n, const double *d, const double *e, double x)
{
    long cnt = 0;
    double bmax = 0.0;
    for (int i = 0; i < n; ++i) bmax = fmax(bmax, fabs(d[i]));
    for (int i = 0; i + 1 < n; ++i) bmax = fmax(bmax, fabs(e[i]));
    double pivmin = fmax(bmax * bmax * 1e-300, 1e-300);
    double q = -x;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) ++cnt;
    for (int i = 1; i < 2 * n; ++i) {
        int j = i - 1;
        double b = (j % 2 == 0) ? d[j / 2] : e[j / 2];
        q = -x - b * b / q;
        if (fabs(q) < pivmin) q = -pivmin;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

/*
 * k-th largest singular value (k = 0 .. n-1) by bisection on Sturm counts:
 * #(s_i < x) = count(x) - n for x > 0.  Stops when the bracket is below
 * 2 eps of its upper end (or absolute width 1e-300).
 */
double oracle_sturm_sigma(int n, const double *d, const double *e, int k)
{
    double hi = 0.0;
    for (int i = 0; i < n; ++i) {                 /* Gershgorin bound on |T| */
        double a = fabs(d[i]);
        double b = (i > 0) ? fabs(e[i - 1]) : 0.0;
        double c = (i + 1 < n) ? fabs(e[i]) : 0.0;
        hi = fmax(hi, fmax(a + b, a + c));
    }
    hi = hi * (1.0 + 4.0 * ORC_EPS) + 1e-300;
    double lo = 0.0;
    long want_below = (long)(n - 1 - k);          /* number of s_i below the target */
    for (int it = 0; it < 4000; ++it) {
        double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        if (hi - lo <= 2.0 * ORC_EPS * hi) break;
        long below = oracle_sturm_count(n, d, e, mid) - n;
        if (below > want_below) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

/*
 * ||B V - U diag(s)||_F / ||B||_F with V = VT^T, using that row r of B has
 * only d[r] (column r) and e[r] (column r+1).  O(n^2).
 */
double oracle_residual(int n, const double *d, const double *e, const double *s,
                       const double *U, int ldu, const double *VT, int ldvt)
{
    /* The ratio does not change when B and S are scaled by the same power of
     * two (exact), so both are taken as d 2^-k, e 2^-k, s 2^-k with 2^k <=
     * max|d, e| < 2^(k+1): the sums of squares then stay inside the exponent
     * range for entries near either end of it. */
    double mx = 0.0;
    for (int i = 0; i < n; ++i) mx = fmax(mx, fabs(d[i]));
    for (int i = 0; i + 1 < n; ++i) mx = fmax(mx, fabs(e[i]));
    const int k = (mx > 0.0 && isfinite(mx)) ? ilogb(mx) : 0;
    double *ds = (double *)malloc(sizeof(double) * (size_t)(3 * n + 1));
    if (!ds) return NAN;
    double *es = ds + n, *ss = es + n;
    for (int i = 0; i < n; ++i) {
        ds[i] = ldexp(d[i], -k);
        es[i] = (i + 1 < n) ? ldexp(e[i], -k) : 0.0;
        ss[i] = ldexp(s[i], -k);
    }
    double num = 0.0, den = 0.0;
    for (int i = 0; i < n; ++i) den += ds[i] * ds[i];
    for (int i = 0; i + 1 < n; ++i) den += es[i] * es[i];
    for (int c = 0; c < n; ++c) {                 /* column c: B v_c - s_c u_c */
        for (int r = 0; r < n; ++r) {
            double bv = ds[r] * VT[(size_t)r * ldvt + c];
            if (r + 1 < n) bv += es[r] * VT[(size_t)(r + 1) * ldvt + c];
            double t = bv - ss[c] * U[(size_t)c * ldu + r];
            num += t * t;
        }
    }
    free(ds);
    return den > 0.0 ? sqrt(num / den) : sqrt(num);
}
