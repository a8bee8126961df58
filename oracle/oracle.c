/*
 * oracle.c -- plain, slow CPU reference for the block-step Hermite direct N-body
 * method (Berczik, Spurzem et al., "Up to 700k GPU cores, Kepler, and the
 * Exascale future for simulations of star clusters around black holes").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker the CUDA path is compared
 * against.  Only the test suite, the package smoke check and the benchmark's CPU
 * baseline may load it; the product path never calls it.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * What the paper states (abstract; "Codes description"): direct summation of the
 * Newtonian gravitational forces between all particles, individual hierarchical
 * ("block") time-steps, and Hermite integration of 4th, 6th and 8th order.  The
 * paper prints no formulas; it defers them to its phi-GPU reference.  Every
 * formula below is therefore the textbook reading of those named methods:
 *
 *   force      exact Plummer-softened direct sum and its time derivatives,
 *              derived by differentiating A = m r / R^3 along the orbit;
 *   predictor  Taylor series in every derivative the particle holds;
 *   corrector  two-point Hermite (Obreschkoff) quadrature of order p;
 *   interp     the unique Hermite polynomial matching acc derivatives 0..p/2-1
 *              at both ends of a step (solved here as a linear system);
 *   time step  generalised Aarseth criterion, quantised to powers of two that
 *              stay commensurate with the block time;
 *   energy     kinetic plus softened pairwise potential energy.
 *
 * Precision: inputs and outputs are double; pairwise terms and every sum are
 * formed in long double (x87 80-bit) so that the oracle's own rounding error is
 * negligible against the double-precision path it checks.
 *
 * Layout: vectors are row-major [n][3]; derivative stacks are [n][6][3] holding
 * a, j(erk), s(nap), c(rackle), d4 = a^(4), d5 = a^(5).  Pair softening is
 * eps_ij^2 = max(eps_i^2, eps_j^2).
 *
 * Return codes: 0 ok, -1 bad argument, -4 time step below dt_min, -5 capacity of
 * an output log exceeded.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef long double ld;

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_DT_UNDERFLOW (-4)
#define ORC_ERR_CAPACITY (-5)

/* ------------------------------------------------------------------------- */
/* Force: direct summation over all j != i (abstract; "Codes description").   */
/* For a pair with r = x_j - x_i, v = v_j - v_i, a = a_j - a_i, k = j_j - j_i  */
/* (predicted values), R^2 = r.r + eps_ij^2:                                  */
/*   A = m_j r / R^3                                                          */
/*   J = dA/dt = m_j v / R^3 - 3 alpha A,         alpha = r.v / R^2            */
/*   S = dJ/dt = m_j a / R^3 - 6 alpha J - 3 beta A,                           */
/*               beta  = (v.v + r.a)/R^2 + alpha^2                             */
/*   C = dS/dt = m_j k / R^3 - 9 alpha S - 9 beta J - 3 gamma A,               */
/*               gamma = (3 v.a + r.k)/R^2 + alpha (3 beta - 4 alpha^2)        */
/*   phi = -m_j / R                                                            */
/* Order 4 uses A, J; order 6 adds S; order 8 adds C.                          */
/* ------------------------------------------------------------------------- */
static ld norm3l(const ld* p)
{
    return sqrtl(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
}

/* absum receives sum_j |A_ij|, |J_ij|, |S_ij|, |C_ij|, |phi_ij|: the size of
   the terms each total is made of, i.e. its condition scale; absum[5] is
   B = sum_j m_j / R_ij^2 (>= sum_j |A_ij|), the acc scale the time step uses. */
static void force_one(int64_t n, const double* m, const double* eps2,
                      const double* x, const double* v, const double* a, const double* jk,
                      int order, int64_t i, ld A[3], ld J[3], ld S[3], ld C[3], ld* phi, ld absum[6])
{
    for (int k = 0; k < 3; k++) { A[k] = 0; J[k] = 0; S[k] = 0; C[k] = 0; }
    for (int k = 0; k < 6; k++) absum[k] = 0;
    *phi = 0;
    for (int64_t j = 0; j < n; j++) {
        if (j == i) continue;
        ld r[3], vv[3], aa[3], kk[3];
        for (int k = 0; k < 3; k++) {
            r[k] = (ld)x[3 * j + k] - (ld)x[3 * i + k];
            vv[k] = (ld)v[3 * j + k] - (ld)v[3 * i + k];
            aa[k] = (order >= 6) ? (ld)a[3 * j + k] - (ld)a[3 * i + k] : 0;
            kk[k] = (order >= 8) ? (ld)jk[3 * j + k] - (ld)jk[3 * i + k] : 0;
        }
        ld e2 = (ld)(eps2[i] > eps2[j] ? eps2[i] : eps2[j]);
        ld R2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + e2;
        if (!(R2 > 0)) continue; /* coincident unsoftened pair: no defined force */
        ld R = sqrtl(R2);
        ld q = (ld)m[j] / (R2 * R);
        ld rv = r[0] * vv[0] + r[1] * vv[1] + r[2] * vv[2];
        ld vsq = vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2];
        ld ra = r[0] * aa[0] + r[1] * aa[1] + r[2] * aa[2];
        ld va = vv[0] * aa[0] + vv[1] * aa[1] + vv[2] * aa[2];
        ld rk = r[0] * kk[0] + r[1] * kk[1] + r[2] * kk[2];
        ld alpha = rv / R2;
        ld beta = (vsq + ra) / R2 + alpha * alpha;
        ld gamma = (3 * va + rk) / R2 + alpha * (3 * beta - 4 * alpha * alpha);
        ld pA[3], pJ[3], pS[3], pC[3];
        for (int k = 0; k < 3; k++) {
            pA[k] = q * r[k];
            pJ[k] = q * vv[k] - 3 * alpha * pA[k];
            pS[k] = q * aa[k] - 6 * alpha * pJ[k] - 3 * beta * pA[k];
            pC[k] = q * kk[k] - 9 * alpha * pS[k] - 9 * beta * pJ[k] - 3 * gamma * pA[k];
            A[k] += pA[k];
            J[k] += pJ[k];
            S[k] += pS[k];
            C[k] += pC[k];
        }
        *phi -= (ld)m[j] / R;
        absum[0] += norm3l(pA);
        absum[1] += norm3l(pJ);
        absum[2] += norm3l(pS);
        absum[3] += norm3l(pC);
        absum[4] += (ld)m[j] / R;
        absum[5] += (ld)m[j] / R2;
    }
}

int orc_force(int64_t n, const double* m, const double* eps2,
              const double* x, const double* v, const double* a, const double* jk,
              int order, int64_t n_act, const int32_t* idx,
              double* acc, double* jerk, double* snap, double* crackle, double* pot,
              double* absum, int nthreads)
{
    if (n < 0 || n_act < 0 || !(order == 4 || order == 6 || order == 8)) return ORC_ERR_ARG;
    if (order >= 6 && !a) return ORC_ERR_ARG;
    if (order >= 8 && !jk) return ORC_ERR_ARG;
    for (int64_t p = 0; p < n_act; p++)
        if (idx[p] < 0 || idx[p] >= n) return ORC_ERR_ARG;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int64_t p = 0; p < n_act; p++) {
        ld A[3], J[3], S[3], C[3], phi, ab[6];
        force_one(n, m, eps2, x, v, a, jk, order, idx[p], A, J, S, C, &phi, ab);
        if (absum)
            for (int k = 0; k < 6; k++) absum[6 * p + k] = (double)ab[k];
        for (int k = 0; k < 3; k++) {
            if (acc) acc[3 * p + k] = (double)A[k];
            if (jerk) jerk[3 * p + k] = (double)J[k];
            if (snap) snap[3 * p + k] = (double)S[k];
            if (crackle) crackle[3 * p + k] = (double)C[k];
        }
        if (pot) pot[p] = (double)phi;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Energy: E = sum 1/2 m v^2 - sum_{i<j} m_i m_j / sqrt(r^2 + eps_ij^2).      */
/* ------------------------------------------------------------------------- */
int orc_energy(int64_t n, const double* m, const double* eps2, const double* x, const double* v,
               double* ekin, double* epot, int nthreads)
{
    if (n < 0) return ORC_ERR_ARG;
    ld k = 0, w = 0;
    for (int64_t i = 0; i < n; i++) {
        ld v2 = 0;
        for (int c = 0; c < 3; c++) v2 += (ld)v[3 * i + c] * (ld)v[3 * i + c];
        k += 0.5L * (ld)m[i] * v2;
    }
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : w) num_threads(nthreads)
#endif
    for (int64_t i = 0; i < n; i++) {
        ld wi = 0;
        for (int64_t j = i + 1; j < n; j++) {
            ld r2 = 0;
            for (int c = 0; c < 3; c++) {
                ld d = (ld)x[3 * j + c] - (ld)x[3 * i + c];
                r2 += d * d;
            }
            r2 += (ld)(eps2[i] > eps2[j] ? eps2[i] : eps2[j]);
            if (r2 > 0) wi -= (ld)m[i] * (ld)m[j] / sqrtl(r2);
        }
        w += wi;
    }
    *ekin = (double)k;
    *epot = (double)w;
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Predictor: Taylor series to the block time using every derivative held.    */
/* Number of acc derivatives (a, j, s, c, d4, d5) that enter, per order:       */
/*   order 4: x and v use a, j, s, c   (s, c interpolated at the last step)    */
/*   order 6: x, v and a use a, j, s, c                                        */
/*   order 8: x, v, a and jerk use a, j, s, c, d4, d5                          */
/* Written as sum_k y^(k) dt^k / k!, the plain definition.                     */
/* ------------------------------------------------------------------------- */
static int pred_nd(int order) { return order == 8 ? 6 : 4; }

static ld fact(int k)
{
    ld f = 1;
    for (int i = 2; i <= k; i++) f *= i;
    return f;
}

/* y^(0) = base, y^(1) = first, then the acc-derivative stack starting at d0. */
static double taylor(double base, const double* first, const double* d, int nd_used, int comp, ld dt)
{
    ld s = base;
    int k = 1;
    if (first) {
        s += (ld)first[comp] * dt;
        k = 2;
    }
    for (int q = 0; q < nd_used; q++, k++) s += (ld)d[3 * q + comp] * powl(dt, k) / fact(k);
    return (double)s;
}

int orc_predict(int64_t n, int order, double t, const double* ti,
                const double* x, const double* v, const double* d,
                double* xp, double* vp, double* ap, double* jp)
{
    if (n < 0 || !(order == 4 || order == 6 || order == 8)) return ORC_ERR_ARG;
    int nd = pred_nd(order);
    for (int64_t i = 0; i < n; i++) {
        ld dt = (ld)t - (ld)ti[i];
        const double* di = d + 18 * i;
        for (int c = 0; c < 3; c++) {
            /* x: x + v dt + sum_{k>=2} d_{k-2} dt^k / k! */
            xp[3 * i + c] = taylor(x[3 * i + c], v + 3 * i, di, nd, c, dt);
            /* v: v + sum_{k>=1} d_{k-1} dt^k / k! */
            vp[3 * i + c] = taylor(v[3 * i + c], NULL, di, nd, c, dt);
            if (ap) ap[3 * i + c] = order >= 6 ? taylor(di[c], NULL, di + 3, nd - 1, c, dt) : di[c];
            if (jp) jp[3 * i + c] = order >= 8 ? taylor(di[3 + c], NULL, di + 6, nd - 2, c, dt) : di[3 + c];
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Corrector: two-point Hermite quadrature of order p for x' = v, v' = a.      */
/*   p=4: y1 = y0 + h/2 (f0+f1) - h^2/12 (f1'-f0')                             */
/*   p=6: y1 = y0 + h/2 (f0+f1) - h^2/10 (f1'-f0') + h^3/120 (f0''+f1'')       */
/*   p=8: y1 = y0 + h/2 (f0+f1) - 3h^2/28 (f1'-f0') + h^3/84 (f0''+f1'')       */
/*                                                  - h^4/1680 (f1'''-f0''')   */
/* v uses f = a (f' = j, ...); x uses f = v (f' = a, ...) with the corrected   */
/* v1.  D0/D1 hold the acc derivatives a, j, s, c at t0 and t1 ([4][3]).       */
/* ------------------------------------------------------------------------- */
static ld hermite_quad(int order, ld h, const ld f0[4], const ld f1[4])
{
    if (order == 4) return h / 2 * (f0[0] + f1[0]) - h * h / 12 * (f1[1] - f0[1]);
    if (order == 6)
        return h / 2 * (f0[0] + f1[0]) - h * h / 10 * (f1[1] - f0[1]) + h * h * h / 120 * (f0[2] + f1[2]);
    return h / 2 * (f0[0] + f1[0]) - 3 * h * h / 28 * (f1[1] - f0[1]) + h * h * h / 84 * (f0[2] + f1[2])
           - h * h * h * h / 1680 * (f1[3] - f0[3]);
}

int orc_correct(int order, double h, const double* x0, const double* v0,
                const double* D0, const double* D1, double* x1, double* v1)
{
    if (!(order == 4 || order == 6 || order == 8)) return ORC_ERR_ARG;
    for (int c = 0; c < 3; c++) {
        ld fa0[4], fa1[4], fv0[4], fv1[4];
        for (int q = 0; q < 4; q++) {
            fa0[q] = D0[3 * q + c];
            fa1[q] = D1[3 * q + c];
        }
        ld vnew = (ld)v0[c] + hermite_quad(order, h, fa0, fa1);
        fv0[0] = v0[c];
        fv1[0] = vnew;
        for (int q = 1; q < 4; q++) {
            fv0[q] = D0[3 * (q - 1) + c];
            fv1[q] = D1[3 * (q - 1) + c];
        }
        ld xnew = (ld)x0[c] + hermite_quad(order, h, fv0, fv1);
        v1[c] = (double)vnew;
        x1[c] = (double)xnew;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Interpolation: acc(tau) = sum_{k<2mm} c_k tau^k / k!, mm = p/2.  The mm     */
/* derivatives at tau = 0 give c_0..c_{mm-1}; the mm derivatives at tau = h    */
/* give a linear system for c_mm..c_{2mm-1}, solved by Gaussian elimination    */
/* with partial pivoting.  Output: derivatives mm..2mm-1 at tau = h.           */
/* D0, D1: [mm][3]; out: [mm][3].                                               */
/* ------------------------------------------------------------------------- */
int orc_interp(int mm, double h, const double* D0, const double* D1, double* out)
{
    if (mm < 1 || mm > 4 || !(h > 0)) return ORC_ERR_ARG;
    for (int c = 0; c < 3; c++) {
        ld M[4][5];
        /* row r: derivative r at tau=h of sum_k c_k tau^k/k!  =  D1[r]        */
        /* known part: sum_{k<mm, k>=r} c_k h^(k-r)/(k-r)!                      */
        for (int r = 0; r < mm; r++) {
            ld rhs = D1[3 * r + c];
            for (int k = r; k < mm; k++) rhs -= (ld)D0[3 * k + c] * powl(h, k - r) / fact(k - r);
            for (int k = mm; k < 2 * mm; k++) M[r][k - mm] = powl(h, k - r) / fact(k - r);
            M[r][mm] = rhs;
        }
        for (int col = 0; col < mm; col++) {
            int piv = col;
            for (int r = col + 1; r < mm; r++)
                if (fabsl(M[r][col]) > fabsl(M[piv][col])) piv = r;
            if (piv != col)
                for (int k = 0; k <= mm; k++) {
                    ld t = M[col][k];
                    M[col][k] = M[piv][k];
                    M[piv][k] = t;
                }
            for (int r = 0; r < mm; r++) {
                if (r == col) continue;
                ld f = M[r][col] / M[col][col];
                for (int k = col; k <= mm; k++) M[r][k] -= f * M[col][k];
            }
        }
        ld cc[8];
        for (int k = 0; k < mm; k++) cc[k] = D0[3 * k + c];
        for (int k = mm; k < 2 * mm; k++) cc[k] = M[k - mm][mm] / M[k - mm][k - mm];
        for (int q = mm; q < 2 * mm; q++) {
            ld s = 0;
            for (int k = q; k < 2 * mm; k++) s += cc[k] * powl(h, k - q) / fact(k - q);
            out[3 * (q - mm) + c] = (double)s;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Time step.                                                                  */
/* Criterion, D = acc derivatives a^(0..p-1) at t1 ([p][3]):                   */
/*   p = 4: dt = sqrt(eta (|a||a2| + |a1|^2) / (|a1||a3| + |a2|^2))            */
/*   p = 6, 8: dt = eta [(sqrt(|a||a2|) + |a1|) /                              */
/*                       (sqrt(|a(p-3)||a(p-1)|) + |a(p-2)|)]^(1/(p-3))        */
/* A zero denominator gives an unbounded step (limited by the quantiser).      */
/* ------------------------------------------------------------------------- */
/* The step decides an integer (a power of two), so it is taken in double, the
   precision of the device path; the acc derivatives it reads are doubles. */
static double norm3d(const double* p)
{
    return sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
}

static double criterion_from_norms(int order, double eta, const double* n)
{
    if (order == 4) {
        double num = n[0] * n[2] + n[1] * n[1], den = n[1] * n[3] + n[2] * n[2];
        if (!(den > 0)) return INFINITY;
        return sqrt(eta * num / den);
    }
    int p = order;
    double num = sqrt(n[0] * n[2]) + n[1], den = sqrt(n[p - 3] * n[p - 1]) + n[p - 2];
    if (!(den > 0)) return INFINITY;
    return eta * pow(num / den, 1.0 / (p - 3));
}

double orc_dt_criterion(int order, double eta, const double* D)
{
    double n[8];
    for (int k = 0; k < order; k++) n[k] = norm3d(D + 3 * k);
    return criterion_from_norms(order, eta, n);
}

/* Noise floor of the interpolated derivatives (reading for reduced-precision
   forces): the new derivatives mm..2mm-1 are linear in the inputs L_r (held,
   at t0) and R_r (new force, at t1), r < mm.  If each input carries relative
   rounding eps[r], derivative k carries at most
       N_k = sum_r |dd_k/dL_r| eps[r] |L_r| + |dd_k/dR_r| eps[r] |R_r| ,
   the partial derivatives read off this oracle's own interpolant by feeding
   it unit inputs.  N[q] is the floor of derivative mm + q. */
int orc_noise_floor(int mm, double h, const double* D0, const double* D1, const double* eps, double* N)
{
    if (mm < 1 || mm > 4 || !(h > 0)) return ORC_ERR_ARG;
    for (int q = 0; q < mm; q++) N[q] = 0;
    for (int r = 0; r < mm; r++) {
        for (int side = 0; side < 2; side++) {
            double U0[12] = {0}, U1[12] = {0}, out[12];
            (side == 0 ? U0 : U1)[3 * r] = 1.0;
            int rc = orc_interp(mm, h, U0, U1, out);
            if (rc) return rc;
            double mag = norm3d((side == 0 ? D0 : D1) + 3 * r);
            for (int q = 0; q < mm; q++) N[q] += fabs(out[3 * q]) * eps[r] * mag;
        }
    }
    return ORC_OK;
}

/* Step criterion after a step of length h: D0 = held derivatives at t0 (rows
   0..mm-1), Dfull = a^(0..2mm-1) at t1 (the first mm from the force, the rest
   interpolated), bacc = sum_j m_j/R_ij^2 of the new force.  Interpolated norms
   are taken net of their noise floor, the input precisions eps scaled by the
   conditioning kappa = max(1, bacc / |a|). */
double orc_dt_criterion_floored(int order, double eta, double h, const double* D0, const double* Dfull,
                                const double* eps, double bacc)
{
    int mm = order / 2;
    double n[8], N[4];
    for (int k = 0; k < 2 * mm; k++) n[k] = norm3d(Dfull + 3 * k);
    if (!(eps[0] > 0 || eps[1] > 0 || eps[2] > 0 || eps[3] > 0)) return criterion_from_norms(order, eta, n);
    double kappa = n[0] > 0 ? bacc / n[0] : 1.0;
    if (!(kappa > 1.0)) kappa = 1.0;
    double ek[4];
    for (int r = 0; r < 4; r++) ek[r] = eps[r] * kappa;
    if (orc_noise_floor(mm, h, D0, Dfull, ek, N)) return NAN;
    for (int q = 0; q < mm; q++) {
        double f = n[mm + q] - N[q];
        n[mm + q] = f > 0 ? f : 0;
    }
    return criterion_from_norms(order, eta, n);
}

/* Largest power-of-two fraction of dt_max that is <= lim, then halved until   */
/* t1 is a multiple of it.  Returns 0 (and *dt_out) or ORC_ERR_DT_UNDERFLOW.    */
int orc_dt_quantise(double lim, double t1, double dt_max, double dt_min, double* dt_out)
{
    double dt = dt_max;
    while (dt > lim && dt >= dt_min) dt *= 0.5;
    while (fmod(t1, dt) != 0.0 && dt >= dt_min) dt *= 0.5;
    *dt_out = dt;
    if (dt < dt_min) return ORC_ERR_DT_UNDERFLOW;
    return ORC_OK;
}

/* Startup step at t = 0 (no history): eta_s |a| / |j|.                        */
double orc_dt_startup(double eta_s, const double* a, const double* j)
{
    double na = norm3d(a), nj = norm3d(j);
    if (!(nj > 0)) return INFINITY;
    return eta_s * na / nj;
}

/* ------------------------------------------------------------------------- */
/* Block scheduler: t_blk = min_i (t_i + dt_i); active = {i : t_i + dt_i ==    */
/* t_blk}, ascending.  All times are dyadic, so the sums are exact.            */
/* ------------------------------------------------------------------------- */
int orc_next_block(int64_t n, const double* ti, const double* dti, double* t_blk,
                   int32_t* idx, int64_t* n_act)
{
    if (n < 1) return ORC_ERR_ARG;
    double tmin = INFINITY;
    for (int64_t i = 0; i < n; i++)
        if (ti[i] + dti[i] < tmin) tmin = ti[i] + dti[i];
    int64_t k = 0;
    for (int64_t i = 0; i < n; i++)
        if (ti[i] + dti[i] == tmin) idx[k++] = (int32_t)i;
    *t_blk = tmin;
    *n_act = k;
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Integrator: individual block time-steps with the Hermite scheme.            */
/* State (all caller-owned, updated in place):                                  */
/*   x, v [n][3]; d [n][6][3] = a, j, s, c, d4, d5; t, dt [n]; pot [n]          */
/* init != 0: start from (x, v) at t = 0: full force, startup step.             */
/* Then block steps until the next block time would exceed t_end.              */
/* The log (if non-NULL) records each block's time, size and active indices.   */
/* ------------------------------------------------------------------------- */
typedef struct {
    double eta, eta_s, dt_max, dt_min, t_end;
    int order, nthreads, init;
    double noise[4]; /* relative precision of acc, jerk, snap, crackle (0: exact) */
} orc_params;

int orc_integrate(int64_t n, const double* m, const double* eps2,
                  double* x, double* v, double* d, double* t, double* dt, double* pot,
                  const orc_params* P,
                  int64_t log_cap_blocks, double* log_t, int64_t* log_nact,
                  int64_t log_cap_idx, int32_t* log_idx, int64_t* n_blocks_out)
{
    int order = P->order;
    if (n < 1 || !(order == 4 || order == 6 || order == 8)) return ORC_ERR_ARG;
    int mm = order / 2;                  /* acc derivatives produced by the force */
    int rc = ORC_OK;
    int64_t nb = 0, nidx = 0;
    double* xp = malloc(sizeof(double) * 3 * n);
    double* vp = malloc(sizeof(double) * 3 * n);
    double* ap = malloc(sizeof(double) * 3 * n);
    double* jp = malloc(sizeof(double) * 3 * n);
    double* F = malloc(sizeof(double) * 12 * n); /* new a, j, s, c per active */
    double* ph = malloc(sizeof(double) * n);
    double* ab = malloc(sizeof(double) * 6 * n);
    int32_t* idx = malloc(sizeof(int32_t) * n);
    if (!xp || !vp || !ap || !jp || !F || !ph || !ab || !idx) {
        rc = ORC_ERR_ARG;
        goto done;
    }

    if (P->init) {
        for (int64_t i = 0; i < n; i++) {
            idx[i] = (int32_t)i;
            t[i] = 0.0;
            for (int q = 0; q < 18; q++) d[18 * i + q] = 0.0;
        }
        /* forces at t = 0 from the initial positions and velocities; the
           predicted acc/jerk of the j-particles are not known yet, so the
           start-up derivatives are built order by order: a, j first, then s
           (needs a_j), then c (needs a_j and jerk_j). */
        for (int pass = 0; pass < (order == 4 ? 1 : order == 6 ? 2 : 3); pass++) {
            int po = pass == 0 ? 4 : pass == 1 ? 6 : 8;
            for (int64_t i = 0; i < n; i++)
                for (int c = 0; c < 3; c++) {
                    ap[3 * i + c] = d[18 * i + c];
                    jp[3 * i + c] = d[18 * i + 3 + c];
                }
            rc = orc_force(n, m, eps2, x, v, ap, jp, po, n, idx, F, F + 3 * n, F + 6 * n, F + 9 * n, ph, NULL,
                           P->nthreads);
            if (rc) goto done;
            for (int64_t i = 0; i < n; i++)
                for (int c = 0; c < 3; c++) {
                    d[18 * i + c] = F[3 * i + c];
                    d[18 * i + 3 + c] = F[3 * n + 3 * i + c];
                    if (po >= 6) d[18 * i + 6 + c] = F[6 * n + 3 * i + c];
                    if (po >= 8) d[18 * i + 9 + c] = F[9 * n + 3 * i + c];
                }
        }
        for (int64_t i = 0; i < n; i++) {
            pot[i] = ph[i];
            double lim = orc_dt_startup(P->eta_s, d + 18 * i, d + 18 * i + 3);
            rc = orc_dt_quantise(lim, 0.0, P->dt_max, P->dt_min, &dt[i]);
            if (rc) goto done;
        }
    }

    for (;;) {
        double tb;
        int64_t na;
        orc_next_block(n, t, dt, &tb, idx, &na);
        if (tb > P->t_end) break;
        if (log_t) {
            if (nb >= log_cap_blocks) {
                rc = ORC_ERR_CAPACITY;
                goto done;
            }
            log_t[nb] = tb;
            log_nact[nb] = na;
        }
        if (log_idx) {
            if (nidx + na > log_cap_idx) {
                rc = ORC_ERR_CAPACITY;
                goto done;
            }
            memcpy(log_idx + nidx, idx, sizeof(int32_t) * na);
            nidx += na;
        }
        nb++;
        rc = orc_predict(n, order, tb, t, x, v, d, xp, vp, ap, jp);
        if (rc) goto done;
        rc = orc_force(n, m, eps2, xp, vp, ap, jp, order, na, idx, F, F + 3 * n, F + 6 * n, F + 9 * n, ph, ab,
                       P->nthreads);
        if (rc) goto done;
        for (int64_t p = 0; p < na; p++) {
            int64_t i = idx[p];
            double h = tb - t[i];
            double D0[12], D1[12];
            for (int q = 0; q < 4; q++)
                for (int c = 0; c < 3; c++) {
                    D0[3 * q + c] = d[18 * i + 3 * q + c];
                    D1[3 * q + c] = (q < mm) ? F[(size_t)q * 3 * n + 3 * p + c] : 0.0;
                }
            /* derivatives mm..2mm-1 at t1 from the Hermite interpolant */
            double hi[12];
            rc = orc_interp(mm, h, D0, D1, hi);
            if (rc) goto done;
            double Dfull[24]; /* a^(0..2mm-1) at t1 */
            for (int q = 0; q < mm; q++)
                for (int c = 0; c < 3; c++) Dfull[3 * q + c] = D1[3 * q + c];
            for (int q = 0; q < mm; q++)
                for (int c = 0; c < 3; c++) Dfull[3 * (mm + q) + c] = hi[3 * q + c];
            /* corrector: needs a..c at both ends; the order-4 rule only reads a, j */
            double D1c[12];
            for (int q = 0; q < 4; q++)
                for (int c = 0; c < 3; c++) D1c[3 * q + c] = Dfull[3 * q + c];
            double x1[3], v1[3];
            orc_correct(order, h, x + 3 * i, v + 3 * i, D0, D1c, x1, v1);
            double crit = orc_dt_criterion_floored(order, P->eta, h, D0, Dfull, P->noise, ab[6 * p + 5]);
            double lim = crit;
            if (2.0 * h < lim) lim = 2.0 * h;
            double dtn;
            rc = orc_dt_quantise(lim, tb, P->dt_max, P->dt_min, &dtn);
            if (rc) goto done;
            for (int c = 0; c < 3; c++) {
                x[3 * i + c] = x1[c];
                v[3 * i + c] = v1[c];
            }
            /* held derivatives: a, j, s, c, d4, d5 at t1 (2mm of them, capped at 6) */
            for (int q = 0; q < 6; q++)
                for (int c = 0; c < 3; c++) d[18 * i + 3 * q + c] = (q < 2 * mm) ? Dfull[3 * q + c] : 0.0;
            t[i] = tb;
            dt[i] = dtn;
            pot[i] = ph[p];
        }
    }
done:
    if (n_blocks_out) *n_blocks_out = nb;
    free(xp);
    free(vp);
    free(ap);
    free(jp);
    free(F);
    free(ph);
    free(ab);
    free(idx);
    return rc;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
