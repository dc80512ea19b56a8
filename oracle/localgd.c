/*
 * ORACLE — test infrastructure only.  Plain, slow, single-threaded FP64 reference
 * of the local diffusion process of "Faster Local Solvers for Graph Diffusion
 * Equations" (arXiv 2410.21634).  Only tests, the package smoke check and the CPU
 * baseline of the benchmark may load it; the CUDA library never does, and this
 * file shares no code with it.
 *
 * Convention (unit source mass; Eq. local-gd divided by alpha, Section 3.3):
 *   PPR  : r0 = e_s, x0 = 0; active u:  x_u += alpha r_u;  r_v += ((1-alpha) r_u)/d_u, v in N(u)
 *   Katz : r0 = e_s, x0 = 0; active u:  x_u += r_u;        r_v += beta r_u,             v in N(u)
 *   HK   : layered Taylor system (Section 2, heat kernel): layer-t node u active in
 *          round t:  x_u += r_u;  r_{t+1,v} += ((tau/(t+1)) r_u)/d_u;  the last layer N
 *          only moves its residual into x.
 *   active set (all kinds): S_t = { u : r_u != 0 and |r_u| >= fl(fl(theta_t eps) d_u) },
 *   theta_t = 1 for PPR and Katz.
 * Nodes of degree 0 have a zero column in A D^-1 and in A: they move their residual
 * into x and scatter nothing.
 *
 * Floating-point contract (so the CUDA path can be compared round by round):
 * every product, quotient and sum below is one IEEE binary64 operation in the
 * order written; compile with -ffp-contract=off.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

enum { ORC_PPR = 0, ORC_KATZ = 1, ORC_HK = 2 };

/* per-round record: |S_t|, vol(S_t), ||r_S||_1 (Definition 3.1, Theorem 3.5) */
typedef struct {
    int64_t n_active;
    int64_t vol_active;
    double rS_l1;
} orc_round;

typedef struct {
    int64_t rounds;       /* T: first round with S_T empty (or the layer count for HK) */
    int64_t volume;       /* sum_t vol(S_t), Definition 3.1 */
    int64_t pushes;       /* sum_t |S_t| */
    double resid_l1;      /* ||r^(T)||_1 (HK: sum over the layers left behind) */
    double x_l1;          /* ||x^(T)||_1 (before the HK e^-tau scaling) */
    int status;           /* 0 converged, 1 round cap reached, -1 allocation failure */
} orc_solve;

static inline int64_t deg_of(const int64_t *off, int64_t u) { return off[u + 1] - off[u]; }

/*
 * S_t in ascending node id, then the snapshot rho_i = r_{u_i} and r_{u_i} = 0 for
 * every u_i in S_t before anything is scattered (Eq. local-gd is a Jacobi step:
 * the pushed values are those of r^(t)).  Returns |S_t|.
 */
static int64_t select_and_snapshot(int64_t n, const int64_t *off, double eps_theta,
                                   double *r, int32_t *active, double *rho, orc_round *st) {
    int64_t k = 0, vol = 0;
    double l1 = 0.0;
    for (int64_t u = 0; u < n; u++) {
        double thr = eps_theta * (double)deg_of(off, u);
        if (r[u] != 0.0 && fabs(r[u]) >= thr) active[k++] = (int32_t)u;
    }
    for (int64_t i = 0; i < k; i++) {
        int32_t u = active[i];
        rho[i] = r[u];
        r[u] = 0.0;
        vol += deg_of(off, u);
        l1 += fabs(rho[i]);
    }
    if (st) { st->n_active = k; st->vol_active = vol; st->rS_l1 = l1; }
    return k;
}

/* One PPR round of Eq. (local-gd): x <- x + alpha r_S ; r <- r - r_S + (1-alpha) A D^-1 r_S */
int64_t oracle_ppr_round(int64_t n, const int64_t *off, const int32_t *col, double alpha,
                         double eps, double *x, double *r, int32_t *active, double *rho,
                         orc_round *st) {
    const double one_minus_alpha = 1.0 - alpha;
    int64_t k = select_and_snapshot(n, off, eps, r, active, rho, st);
    for (int64_t i = 0; i < k; i++) {
        int32_t u = active[i];
        int64_t d = deg_of(off, u);
        x[u] = x[u] + alpha * rho[i];
        if (d == 0) continue;
        double w = (one_minus_alpha * rho[i]) / (double)d;
        for (int64_t e = off[u]; e < off[u + 1]; e++) r[col[e]] = r[col[e]] + w;
    }
    return k;
}

/* One Katz round of Eq. (local-gd) with Q = I - beta A: x <- x + r_S ; r <- r - r_S + beta A r_S */
int64_t oracle_katz_round(int64_t n, const int64_t *off, const int32_t *col, double beta,
                          double eps, double *x, double *r, int32_t *active, double *rho,
                          orc_round *st) {
    int64_t k = select_and_snapshot(n, off, eps, r, active, rho, st);
    for (int64_t i = 0; i < k; i++) {
        int32_t u = active[i];
        x[u] = x[u] + rho[i];
        double w = beta * rho[i];
        for (int64_t e = off[u]; e < off[u + 1]; e++) r[col[e]] = r[col[e]] + w;
    }
    return k;
}

/*
 * One heat-kernel round t on the layered system (I - S (x) M) v = e_1 (x) e_s with
 * S[t+1, t] = tau/(t+1) and M = A D^-1: the active layer-t nodes move their
 * residual into x and, unless t is the last layer, scatter ((tau/(t+1)) r_u)/d_u to
 * each neighbour's layer-(t+1) residual r_next.  eps_theta = fl(theta_t eps).
 */
int64_t oracle_hk_round(int64_t n, const int64_t *off, const int32_t *col, double tau,
                        int64_t t, int propagate, double eps_theta, double *x, double *r,
                        double *r_next, int32_t *active, double *rho, orc_round *st) {
    const double coef = tau / (double)(t + 1);
    int64_t k = select_and_snapshot(n, off, eps_theta, r, active, rho, st);
    for (int64_t i = 0; i < k; i++) {
        int32_t u = active[i];
        int64_t d = deg_of(off, u);
        x[u] = x[u] + rho[i];
        if (!propagate || d == 0) continue;
        double w = (coef * rho[i]) / (double)d;
        for (int64_t e = off[u]; e < off[u + 1]; e++) r_next[col[e]] = r_next[col[e]] + w;
    }
    return k;
}

/*
 * Generalised propagation (the InstantGNN propagation of Section 4 and its push in the
 * appendix on InstantGNN(LocalGS); beta = 1/2 gives APPNP's D^-1/2 A D^-1/2 of Table 1,
 * beta = 0 gives PPR): f = sum_k alpha (1-alpha)^k M^k e_s with M = D^-beta A D^(beta-1).
 * One LocalGD round: S_t = { u : r_u != 0, |r_u| >= eps d_u^(1-beta) } in ascending id,
 * snapshot and zero r_S, then for u in S_t: x_u += alpha r_u and, for v in N(u) in CSR
 * order, r_v += ((1-alpha) r_u) / (d_u^(1-beta) d_v^beta).
 */
int64_t oracle_gppr_round(int64_t n, const int64_t *off, const int32_t *col, double alpha,
                          double beta, double eps, double *x, double *r, int32_t *active,
                          double *rho, orc_round *st) {
    int64_t k = 0, vol = 0;
    double l1 = 0.0;
    for (int64_t u = 0; u < n; u++) {
        double thr_u = eps * pow((double)deg_of(off, u), 1.0 - beta);
        if (r[u] != 0.0 && fabs(r[u]) >= thr_u) active[k++] = (int32_t)u;
    }
    for (int64_t i = 0; i < k; i++) {
        int32_t u = active[i];
        rho[i] = r[u];
        vol += deg_of(off, u);
        l1 += fabs(rho[i]);
        r[u] = 0.0;
    }
    if (st) { st->n_active = k; st->vol_active = vol; st->rS_l1 = l1; }
    const double keep = 1.0 - alpha;  /* the share 1 - alpha that is propagated */
    for (int64_t i = 0; i < k; i++) {
        int32_t u = active[i];
        int64_t d = deg_of(off, u);
        x[u] += alpha * rho[i];
        if (d == 0) continue;
        double du = pow((double)d, 1.0 - beta);
        for (int64_t e = off[u]; e < off[u + 1]; e++) {
            int32_t v = col[e];
            double dv = pow((double)deg_of(off, v), beta);
            r[v] = r[v] + (keep * rho[i]) / (du * dv);
        }
    }
    return k;
}

/* Generalised propagation from e_seed until the active set is empty (or max_rounds). */
int oracle_gppr_solve(int64_t n, const int64_t *off, const int32_t *col, double alpha, double beta,
                      double eps, int32_t seed, int64_t max_rounds, double *x, orc_round *total,
                      int64_t *rounds_out) {
    double *r = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    int32_t *active = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    double *rho = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!r || !active || !rho) { free(r); free(active); free(rho); return -1; }
    memset(x, 0, sizeof(double) * (size_t)n);
    r[seed] = 1.0;
    int64_t t = 0, vol = 0, pushes = 0;
    for (; t < max_rounds; t++) {
        orc_round st;
        int64_t k = oracle_gppr_round(n, off, col, alpha, beta, eps, x, r, active, rho, &st);
        if (k == 0) break;
        vol += st.vol_active;
        pushes += k;
    }
    double rl1 = 0.0;
    for (int64_t u = 0; u < n; u++) rl1 += fabs(r[u]);
    if (total) { total->n_active = pushes; total->vol_active = vol; total->rS_l1 = rl1; }
    if (rounds_out) *rounds_out = t;
    free(r); free(active); free(rho);
    return t >= max_rounds ? 1 : 0;
}

/*
 * A general power series f = sum_{k=0}^{N} c_k M^k e_s, M = A D^-1, c_k > 0 (Eq. 1 with the
 * coefficients of Table 1, e.g. IPR's theta^k / (theta^k + theta^10)^2): the heat kernel's
 * layered system (Section 2) with layer ratio c_{t+1}/c_t.  Round t: the active layer-t
 * nodes move their residual into x and, unless t = N, scatter ((c_{t+1}/c_t) r_u)/d_u to
 * each neighbour's layer-(t+1) residual.  The result is f ~ c_0 x.
 */
int64_t oracle_series_round(int64_t n, const int64_t *off, const int32_t *col, double ratio,
                            int propagate, double eps_theta, double *x, double *r, double *r_next,
                            int32_t *active, double *rho, orc_round *st) {
    int64_t k = select_and_snapshot(n, off, eps_theta, r, active, rho, st);
    for (int64_t i = 0; i < k; i++) {
        int32_t u = active[i];
        int64_t d = deg_of(off, u);
        x[u] = x[u] + rho[i];
        if (!propagate || d == 0) continue;
        double w = (ratio * rho[i]) / (double)d;
        for (int64_t e = off[u]; e < off[u + 1]; e++) r_next[col[e]] = r_next[col[e]] + w;
    }
    return k;
}

/* psi_t = sum_{j=0}^{N-t} c_{t+j}/c_t: the weight of one unit of layer-t residual */
double oracle_series_psi(const double *c, int64_t N, int64_t t) {
    double psi = 0.0;
    for (int64_t j = 0; j <= N - t; j++) psi += c[t + j] / c[t];
    return psi;
}

/*
 * Threshold scale of layer t: 1/((N+1) c_0 psi_t) (mode 0), which gives
 * 0 <= f_N - c_0 x <= eps d_u at exit (each layer's leftover residual r_t adds at most
 * c_0 psi_t theta_t eps d_u through the reversibility of A D^-1), or 1 (mode 1).
 */
double oracle_series_theta(const double *c, int64_t N, int64_t t, int mode) {
    if (mode == 1) return 1.0;
    return 1.0 / ((double)(N + 1) * c[0] * oracle_series_psi(c, N, t));
}

/* The series solve from e_seed: layers 0..N, x returned already scaled by c_0. */
int oracle_series_solve(int64_t n, const int64_t *off, const int32_t *col, const double *c, int64_t N,
                        double eps, int32_t seed, int mode, int64_t max_rounds, double *x,
                        orc_solve *res) {
    memset(res, 0, sizeof(*res));
    double *r = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *r2 = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    int32_t *active = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    double *rho = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!r || !r2 || !active || !rho) {
        free(r); free(r2); free(active); free(rho);
        res->status = -1;
        return -1;
    }
    memset(x, 0, sizeof(double) * (size_t)n);
    r[seed] = 1.0;
    double retired = 0.0;
    int64_t t = 0;
    for (t = 0; t < max_rounds && t <= N; t++) {
        orc_round st;
        double ratio = t < N ? c[t + 1] / c[t] : 0.0;
        double eps_theta = oracle_series_theta(c, N, t, mode) * eps;
        int64_t k = oracle_series_round(n, off, col, ratio, t < N, eps_theta, x, r, r2, active, rho, &st);
        if (k == 0) break;
        res->volume += st.vol_active;
        res->pushes += st.n_active;
        for (int64_t u = 0; u < n; u++) retired += fabs(r[u]);
        double *tmp = r; r = r2; r2 = tmp;
        memset(r2, 0, sizeof(double) * (size_t)n);
    }
    res->rounds = t;
    res->status = (t >= max_rounds) ? 1 : 0;
    double rl1 = retired, xl1 = 0.0;
    for (int64_t u = 0; u < n; u++) { rl1 += fabs(r[u]); xl1 += fabs(x[u]); }
    res->resid_l1 = rl1;
    res->x_l1 = xl1;
    for (int64_t u = 0; u < n; u++) x[u] = c[0] * x[u];
    free(r); free(r2); free(active); free(rho);
    return res->status;
}

/*
 * Standard (global) gradient descent, the counterpart of LocalGD in the comparison of
 * Section 5 (Table 2, Figure 6): every iteration updates every node, x <- x + c r and
 * r <- M r (PPR: c = alpha, M = (1-alpha) A D^-1; Katz: c = 1, M = beta A), which is the
 * LocalGD round with the threshold at 0 (nodes with r_u = 0 contribute nothing).  It stops
 * when max_u |r_u| / d_u < eps (||D^-1 r||_inf, degree-0 nodes read as degree 1), and its
 * operation count is iterations x nnz (the standard algorithm touches every edge).
 * Returns the number of iterations, or -1 on allocation failure.
 */
int64_t oracle_gd_solve(int64_t n, const int64_t *off, const int32_t *col, int kind, double param,
                        double eps, int32_t seed, int64_t max_iter, double *x) {
    double *r = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    int32_t *active = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    double *rho = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!r || !active || !rho) { free(r); free(active); free(rho); return -1; }
    memset(x, 0, sizeof(double) * (size_t)n);
    r[seed] = 1.0;
    int64_t it = 0;
    for (; it < max_iter; it++) {
        double worst = 0.0;
        for (int64_t u = 0; u < n; u++) {
            int64_t d = deg_of(off, u);
            double q = fabs(r[u]) / (double)(d > 0 ? d : 1);
            if (q > worst) worst = q;
        }
        if (worst < eps) break;
        if (kind == ORC_PPR) oracle_ppr_round(n, off, col, param, 0.0, x, r, active, rho, NULL);
        else oracle_katz_round(n, off, col, param, 0.0, x, r, active, rho, NULL);
    }
    free(r); free(active); free(rho);
    return it;
}

/*
 * LocalCH for PPR (Section 3.3's local Chebyshev method; its PPR updates in the appendix on
 * implementation details), in the unit-mass variables of this file (x estimates f, the
 * paper's D^1/2 r is alpha r).  Chebyshev on Q = I - (1-alpha) D^-1/2 A D^-1/2 with
 * eigenvalues in [alpha, 2 - alpha]: delta_1 = 1 - alpha, delta_{t+1} = 1/(2/(1-alpha) - delta_t).
 * Round 0 pushes S_0 as LocalGD does (xh = alpha r).  Round t >= 1, for u in
 * S_t = { u : r_u != 0, |r_u| >= eps d_u } (ascending id, snapshot rho = r before any scatter):
 *   xh_u = (2 delta_{t+1}/(1-alpha)) alpha rho_u + delta_t delta_{t+1} (x^t - x^{t-1})_u,
 *   x_u += xh_u,  r_u = rho_u - xh_u/alpha,  r_v += ((1-alpha) xh_u/alpha)/d_u for v in N(u),
 * i.e. x += xh_S and r -= Q_w xh_S / alpha with Q_w = I - (1-alpha) A D^-1, which keeps
 * Q_w x / alpha + r = e_s.  The momentum is restricted to S_t; it stops when S_t is empty.
 * Returns the number of rounds (or -1 on allocation failure).
 */
int64_t oracle_localch_solve(int64_t n, const int64_t *off, const int32_t *col, double alpha, double eps,
                             int32_t seed, int64_t max_rounds, double *x, double *r_out, int64_t *volume) {
    double *r = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *dx = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));   /* x^t - x^{t-1} */
    double *dxn = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    int32_t *act = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    double *rho = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *xh = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!r || !dx || !dxn || !act || !rho || !xh) {
        free(r); free(dx); free(dxn); free(act); free(rho); free(xh);
        return -1;
    }
    memset(x, 0, sizeof(double) * (size_t)n);
    r[seed] = 1.0;
    const double c = 1.0 - alpha;
    double delta = c;  /* delta_1 */
    int64_t t = 0, vol = 0;
    for (; t < max_rounds; t++) {
        int64_t k = 0;
        for (int64_t u = 0; u < n; u++) {
            double th = eps * (double)deg_of(off, u);
            if (r[u] != 0.0 && fabs(r[u]) >= th) act[k++] = (int32_t)u;
        }
        if (k == 0) break;
        double dnext = 0.0, g1 = 0.0, g2 = 0.0;
        if (t > 0) {
            dnext = 1.0 / (2.0 / c - delta);
            g1 = (2.0 * dnext) / c;
            g2 = delta * dnext;
        }
        for (int64_t i = 0; i < k; i++) {
            int32_t u = act[i];
            rho[i] = r[u];
            if (t == 0) xh[i] = alpha * rho[i];
            else xh[i] = g1 * (alpha * rho[i]) + g2 * dx[u];
        }
        for (int64_t i = 0; i < k; i++) {
            int32_t u = act[i];
            x[u] = x[u] + xh[i];
            r[u] = rho[i] - xh[i] / alpha;
            dxn[u] = xh[i];
            vol += deg_of(off, u);
        }
        for (int64_t i = 0; i < k; i++) {
            int32_t u = act[i];
            int64_t d = deg_of(off, u);
            if (d == 0) continue;
            double w = (c * (xh[i] / alpha)) / (double)d;
            for (int64_t e = off[u]; e < off[u + 1]; e++) r[col[e]] = r[col[e]] + w;
        }
        /* the next round's momentum is this round's update, zero off S_t */
        double *tmp = dx; dx = dxn; dxn = tmp;
        memset(dxn, 0, sizeof(double) * (size_t)n);
        if (t > 0) delta = dnext;
    }
    if (r_out) memcpy(r_out, r, sizeof(double) * (size_t)n);
    if (volume) *volume = vol;
    free(r); free(dx); free(dxn); free(act); free(rho); free(xh);
    return t;
}

/* ------------------------------------------------------- heat-kernel terms */

/*
 * Number of Taylor terms: the smallest N with e^-tau sum_{k>N} tau^k/k! <= tol
 * (Poisson tail; the heat kernel of Section 2 truncated after N+1 terms).  The
 * tail is summed from its small end so it stays accurate near tol.
 */
int64_t oracle_hk_terms(double tau, double tol) {
    int64_t kmax = (int64_t)(10.0 * tau) + 200;
    double *p = (double *)malloc(sizeof(double) * (size_t)(kmax + 2));
    if (!p) return -1;
    p[0] = exp(-tau);
    for (int64_t k = 0; k < kmax; k++) p[k + 1] = p[k] * tau / (double)(k + 1);
    /* tail[N] = sum_{k=N+1}^{kmax} p_k, accumulated downwards */
    double tail = 0.0;
    int64_t best = kmax;
    for (int64_t N = kmax - 1; N >= 0; N--) {
        tail += p[N + 1];
        if (tail <= tol) best = N; else break;
    }
    free(p);
    return best;
}

/* psi_k(tau) = sum_{j=0}^{N-k} tau^j k!/(k+j)!  (weight of one unit of layer-k residual) */
double oracle_hk_psi(double tau, int64_t N, int64_t k) {
    double s = 0.0, term = 1.0;
    for (int64_t j = 0; j <= N - k; j++) {
        if (j > 0) term = term * (tau / (double)(k + j));
        s += term;
    }
    return s;
}

/*
 * Threshold scale theta_t of layer t.  mode 0: theta_t = e^tau / ((N+1) psi_t(tau)),
 * which bounds the leftover residual's contribution to e^-tau x by eps d_u per layer
 * (error reading of the heat-kernel stop rule); mode 1: theta_t = 1 (the literal
 * |r_u| >= eps d_u rule).
 */
double oracle_hk_theta(double tau, int64_t N, int64_t t, int mode) {
    if (mode == 1) return 1.0;
    return exp(tau) / ((double)(N + 1) * oracle_hk_psi(tau, N, t));
}

/* ----------------------------------------------------------------- solve */


/*
 * LocalGD from the unit source e_s until S_T is empty (or max_rounds rounds).
 * x_out receives x (PPR, Katz) or e^-tau x (HK).  If log is non-NULL it receives
 * one orc_round per round (log_cap entries at most).
 */
int oracle_localgd_solve(int64_t n, const int64_t *off, const int32_t *col, int kind,
                         double param, double eps, int32_t seed, int hk_mode, double hk_tol,
                         int64_t max_rounds, double *x_out, orc_solve *res, orc_round *log,
                         int64_t log_cap) {
    memset(res, 0, sizeof(*res));
    double *x = x_out;
    double *r = (double *)calloc((size_t)n, sizeof(double));
    double *r2 = kind == ORC_HK ? (double *)calloc((size_t)n, sizeof(double)) : NULL;
    int32_t *active = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    double *rho = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!r || !active || !rho || (kind == ORC_HK && !r2)) {
        free(r); free(r2); free(active); free(rho);
        res->status = -1;
        return -1;
    }
    memset(x, 0, sizeof(double) * (size_t)n);
    r[seed] = 1.0;
    int64_t N = kind == ORC_HK ? oracle_hk_terms(param, hk_tol) : 0;
    double retired = 0.0; /* HK: residual mass left behind in finished layers */
    int64_t t = 0;
    for (t = 0; t < max_rounds; t++) {
        orc_round st;
        int64_t k;
        if (kind == ORC_PPR) {
            k = oracle_ppr_round(n, off, col, param, eps, x, r, active, rho, &st);
        } else if (kind == ORC_KATZ) {
            k = oracle_katz_round(n, off, col, param, eps, x, r, active, rho, &st);
        } else {
            if (t > N) break;
            double eps_theta = oracle_hk_theta(param, N, t, hk_mode) * eps;
            k = oracle_hk_round(n, off, col, param, t, t < N, eps_theta, x, r, r2, active,
                                rho, &st);
        }
        if (k == 0) break;
        if (log && t < log_cap) log[t] = st;
        res->volume += st.vol_active;
        res->pushes += st.n_active;
        if (kind == ORC_HK) {
            /* layer t is finished: what is left of it stays behind; layer t+1 becomes current */
            for (int64_t u = 0; u < n; u++) retired += fabs(r[u]);
            double *tmp = r; r = r2; r2 = tmp;
            memset(r2, 0, sizeof(double) * (size_t)n);
        }
    }
    res->rounds = t;
    res->status = (t >= max_rounds) ? 1 : 0;
    double rl1 = retired, xl1 = 0.0;
    for (int64_t u = 0; u < n; u++) { rl1 += fabs(r[u]); xl1 += fabs(x[u]); }
    res->resid_l1 = rl1;
    res->x_l1 = xl1;
    if (kind == ORC_HK) {
        double scale = exp(-param);
        for (int64_t u = 0; u < n; u++) x[u] = scale * x[u];
    }
    free(r); free(r2); free(active); free(rho);
    return res->status;
}

/* Independent solves for several sources, one source per OpenMP thread (CPU baseline). */
int oracle_localgd_solve_many(int64_t n, const int64_t *off, const int32_t *col, int kind,
                              double param, double eps, const int32_t *seeds, int64_t nseeds,
                              int hk_mode, double hk_tol, int64_t max_rounds, double *xs,
                              orc_solve *res) {
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int64_t i = 0; i < nseeds; i++) {
        int s = oracle_localgd_solve(n, off, col, kind, param, eps, seeds[i], hk_mode, hk_tol,
                                     max_rounds, xs + i * n, &res[i], NULL, 0);
        if (s < 0) bad = 1;
    }
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------- FIFO push */

/*
 * Sequential push with a FIFO queue (Algo 1, APPR; AKatz and AHK of Section 2 in
 * the same way): while some queued u has r_u != 0 and |r_u| >= theta eps d_u, save
 * r_u, set it to zero, move it into x and add the weighted share to each
 * neighbour, queueing neighbours that reach their threshold.  Gauss-Seidel order:
 * every push sees the residuals written by the pushes before it.  For HK the queue
 * holds (layer, node) pairs.  Returns the number of pushes, -1 on allocation failure.
 * x_out receives x (PPR, Katz) or e^-tau x (HK); *volume receives sum of d_u pushed.
 */
int64_t oracle_push_fifo(int64_t n, const int64_t *off, const int32_t *col, int kind,
                         double param, double eps, int32_t seed, int hk_mode, double hk_tol,
                         double *x_out, int64_t *volume) {
    int64_t N = kind == ORC_HK ? oracle_hk_terms(param, hk_tol) : 0;
    int64_t L = N + 1; /* residual layers (1 for PPR and Katz) */
    double *r = (double *)calloc((size_t)(n * L), sizeof(double));
    char *inq = (char *)calloc((size_t)(n * L), 1);
    double *eps_theta = (double *)malloc(sizeof(double) * (size_t)L);
    int64_t qcap = n * L + 1;
    int64_t *q = (int64_t *)malloc(sizeof(int64_t) * (size_t)qcap);
    if (!r || !inq || !q || !eps_theta) {
        free(r); free(inq); free(q); free(eps_theta);
        return -1;
    }
    for (int64_t k = 0; k < L; k++)
        eps_theta[k] = (kind == ORC_HK ? oracle_hk_theta(param, N, k, hk_mode) : 1.0) * eps;
    memset(x_out, 0, sizeof(double) * (size_t)n);
    int64_t head = 0, tail = 0, pushes = 0, vol = 0;
    r[seed] = 1.0;
    q[tail++ % qcap] = seed;
    inq[seed] = 1;
    while (head != tail) {
        int64_t id = q[head++ % qcap];
        inq[id] = 0;
        int64_t layer = id / n, u = id % n;
        int64_t d = deg_of(off, u);
        double thr = eps_theta[layer] * (double)d;
        if (!(r[id] != 0.0 && fabs(r[id]) >= thr)) continue;
        double rt = r[id];
        r[id] = 0.0;
        pushes++;
        vol += d;
        double w = 0.0;
        int64_t tgt_layer = layer;
        if (kind == ORC_PPR) {
            x_out[u] = x_out[u] + param * rt;
            if (d == 0) continue;
            w = ((1.0 - param) * rt) / (double)d;
        } else if (kind == ORC_KATZ) {
            x_out[u] = x_out[u] + rt;
            w = param * rt;
        } else {
            x_out[u] = x_out[u] + rt;
            if (layer == N || d == 0) continue;
            w = ((param / (double)(layer + 1)) * rt) / (double)d;
            tgt_layer = layer + 1;
        }
        double vthr = eps_theta[tgt_layer];
        for (int64_t e = off[u]; e < off[u + 1]; e++) {
            int64_t v = col[e];
            int64_t vid = tgt_layer * n + v;
            r[vid] = r[vid] + w;
            if (!inq[vid] && fabs(r[vid]) >= vthr * (double)deg_of(off, v)) {
                inq[vid] = 1;
                q[tail++ % qcap] = vid;
            }
        }
    }
    if (kind == ORC_HK) {
        double scale = exp(-param);
        for (int64_t u = 0; u < n; u++) x_out[u] = scale * x_out[u];
    }
    if (volume) *volume = vol;
    free(r); free(inq); free(q); free(eps_theta);
    return pushes;
}
