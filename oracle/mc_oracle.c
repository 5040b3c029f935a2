/*
 * FP64 CPU oracle for the interface Monte Carlo of the stochastic-deterministic
 * domain decomposition (SDD) mesh generator of Bihlo & Haynes,
 * "Parallel stochastic methods for PDE based grid generation" (arXiv 1310.3435).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference the CUDA
 * path is checked against.  Only tests/, the smoke check and the benchmark's
 * CPU-baseline leg load it.  It shares no code, header or constant table with
 * the CUDA library; both sides implement the published definitions separately.
 *
 * What it computes (paper §2.1-2.2):
 *   The linear Winslow generator  -div(c grad u) = 0  on the unit square
 *   (eq. WinslowTypeGridGenerator, with c = w or c = 1/w, see coef_mode) has the
 *   Feynman-Kac representation  u(x) = E[ u_boundary(X_tau) ]  (eq. ...StochasticSolutionA)
 *   for the Ito diffusion  dX = grad(ln c) dt + sqrt(2) dW  stopped at the first
 *   exit tau from the square.  The expanded form of the PDE (eq. ...Expanded) is
 *   Lap u + grad(ln c).grad u = 0, whose generator fixes the noise scale sqrt(2):
 *   the printed SDE (eq. ...StochasticSolutionB) omits the factor, and the printed
 *   increment "2 sqrt(dt) N(0,1)" (§2.2) is read as sqrt(2 dt) N(0,1).
 *   Paths are advanced with Euler-Maruyama (§2.2), the exit test is applied at
 *   the end of each step (§2.2), the exit point is the intersection of the last
 *   step's segment with the side it crossed, the score is the boundary map at the
 *   exit point by linear interpolation of the per-edge tables, and the per-node
 *   estimate is the sample mean with error ~ N^-1/2 (§2.2).
 *
 * Random numbers (§2.2 uses pseudo-random numbers): Philox4x32-10 of Salmon,
 * Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11),
 * keyed by the 64-bit seed, counter = (step/2, path, node, 0).  Each block of
 * four 32-bit words gives four uniforms U_m = (r_m + 1/2) 2^-32 and, by the
 * Box-Muller transform, the two normal pairs of steps k and k+1 (k even):
 *   step k   : R = sqrt(-2 ln U0), z = (R cos 2 pi U1, R sin 2 pi U1)
 *   step k+1 : R = sqrt(-2 ln U2), z = (R cos 2 pi U3, R sin 2 pi U3)
 *
 * Exponential time stepping (§2.2, after Jansons and Lythe): step k has the
 * random length h_k = dt E_k, E_k = -ln U a unit-mean exponential, so the
 * steps have the density lambda exp(-lambda h) with lambda = 1/dt.  The four
 * lengths of steps 4m .. 4m+3 come from words 0..3 of
 * Philox(counter = (m, path, node, 2)).  Given h_k the update is the
 * Euler-Maruyama one with step h_k, and the boundary test is the exact
 * crossing probability of the step's Brownian bridge over the time h_k (the
 * Brownian-bridge test below with dt replaced by h_k), which is how the
 * exponential steps take their boundary test.
 *
 * Build: plain C99, -O2 -ffp-contract=off, no fast-math (oracle/build.py).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------- Philox -- */
/* Philox4x32-10 as defined in Salmon et al. (SC'11), §4: ten rounds of
 *   (hi0,lo0) = M0 * x0,  (hi1,lo1) = M1 * x2   (32x32 -> 64-bit products)
 *   x' = (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0)
 * with the key advanced by the Weyl constants between rounds. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        x0 = y0;
        x1 = lo1;
        x2 = y2;
        x3 = lo0;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* The four normals of steps k and k+1 (k even) of path `path` at node `node`. */
void oracle_normals(uint64_t seed, uint32_t node, uint32_t path, uint32_t step_pair,
                    double z[4])
{
    uint32_t ctr[4] = {step_pair, path, node, 0u};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t r[4];
    oracle_philox4x32_10(ctr, key, r);
    double u[4];
    for (int m = 0; m < 4; ++m)
        u[m] = ((double)r[m] + 0.5) * 0x1p-32;        /* exact, in (0,1) */
    double ra = sqrt(-2.0 * log(u[0]));
    double rb = sqrt(-2.0 * log(u[2]));
    z[0] = ra * cos(2.0 * M_PI * u[1]);
    z[1] = ra * sin(2.0 * M_PI * u[1]);
    z[2] = rb * cos(2.0 * M_PI * u[3]);
    z[3] = rb * sin(2.0 * M_PI * u[3]);
}

/* Unit-mean exponentials of the lengths of steps 4q .. 4q+3 under exponential
 * time stepping: E = -ln U, U = (r + 1/2) 2^-32 from words 0..3 of
 * Philox(counter = (q, path, node, 2)). */
void oracle_step_lengths(uint64_t seed, uint32_t node, uint32_t path, uint32_t quad,
                         double E[4])
{
    uint32_t ctr[4] = {quad, path, node, 2u};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t r[4];
    oracle_philox4x32_10(ctr, key, r);
    for (int m = 0; m < 4; ++m)
        E[m] = -log(((double)r[m] + 0.5) * 0x1p-32);
}

/* --------------------------------------------------------------- density -- */
/* Density families (shapes of the paper's monitor functions, eqs.
 * MonitorFunctionRunningExample, MackenzieMonitorFunction, and the ring of
 * FiveRingMonitorFunction):
 *   0 BUMPS : params = [nb, (A, cs, ct, ks, kt) x nb]
 *             w = 1 + sum_b A exp(-ks (s-cs)^2 - kt (t-ct)^2)
 *   1 RING  : params = [A, cs, ct, k, r0]
 *             w = 1 + A sech^2(k (r - r0)),  r = |(s,t) - (cs,ct)|
 *   2 RIDGE : params = [A, k, t0, a, f]
 *             w = 1 + A exp(-k (t - t0 - a sin(2 pi f s))^2)
 *   3 TABLE : params = [tn, L(0,0), L(1,0), ..., L(tn-1,tn-1)]: ln w at the
 *             tn x tn nodes (a/(tn-1), b/(tn-1)), row b after row b-1;
 *             w = exp(L), L the bilinear interpolant of the nodes, and
 *             grad ln w = grad L, the interpolant's exact (cellwise) gradient
 * The generator's coefficient is c = w (coef_mode 0) or c = 1/w (coef_mode 1). */

/* Bilinear interpolant L of a table of ln w and its gradient at (s,t); the
 * cell is the one holding (s,t), the last one on the upper sides. */
static void table_L(const double* p, double s, double t, double* L, double* Ls, double* Lt)
{
    int tn = (int)p[0];
    const double* T = p + 1;
    double m = (double)(tn - 1);
    double x = s * m, y = t * m;
    int a = (int)floor(x), b = (int)floor(y);
    if (a > tn - 2) a = tn - 2;
    if (a < 0) a = 0;
    if (b > tn - 2) b = tn - 2;
    if (b < 0) b = 0;
    double fa = x - (double)a, fb = y - (double)b;
    double L00 = T[b * tn + a], L10 = T[b * tn + a + 1];
    double L01 = T[(b + 1) * tn + a], L11 = T[(b + 1) * tn + a + 1];
    *L = (1.0 - fb) * ((1.0 - fa) * L00 + fa * L10) + fb * ((1.0 - fa) * L01 + fa * L11);
    *Ls = ((1.0 - fb) * (L10 - L00) + fb * (L11 - L01)) * m;
    *Lt = ((1.0 - fa) * (L01 - L00) + fa * (L11 - L10)) * m;
}

/* w and grad w at (s,t). */
static void density_w(int family, const double* p, double s, double t,
                      double* w, double* ws, double* wt)
{
    if (family == 3) {
        double L, Ls, Lt;
        table_L(p, s, t, &L, &Ls, &Lt);
        *w = exp(L);
        *ws = *w * Ls;
        *wt = *w * Lt;
    } else if (family == 0) {
        int nb = (int)p[0];
        double acc = 1.0, gs = 0.0, gt = 0.0;
        for (int b = 0; b < nb; ++b) {
            const double* q = p + 1 + 5 * b;
            double A = q[0], cs = q[1], ct = q[2], ks = q[3], kt = q[4];
            double e = A * exp(-ks * (s - cs) * (s - cs) - kt * (t - ct) * (t - ct));
            acc += e;
            gs += e * (-2.0 * ks * (s - cs));
            gt += e * (-2.0 * kt * (t - ct));
        }
        *w = acc; *ws = gs; *wt = gt;
    } else if (family == 1) {
        double A = p[0], cs = p[1], ct = p[2], k = p[3], r0 = p[4];
        double ds = s - cs, dtt = t - ct;
        double r = sqrt(ds * ds + dtt * dtt);
        double u = k * (r - r0);
        double sech = 1.0 / cosh(u);
        double sech2 = sech * sech;
        *w = 1.0 + A * sech2;
        if (r > 0.0) {
            double dwdr = A * (-2.0 * k * sech2 * tanh(u));
            *ws = dwdr * ds / r;
            *wt = dwdr * dtt / r;
        } else {
            *ws = 0.0;
            *wt = 0.0;
        }
    } else {
        double A = p[0], k = p[1], t0 = p[2], a = p[3], f = p[4];
        double v = t - t0 - a * sin(2.0 * M_PI * f * s);
        double e = A * exp(-k * v * v);
        *w = 1.0 + e;
        *wt = e * (-2.0 * k * v);
        *ws = e * (-2.0 * k * v) * (-a * 2.0 * M_PI * f * cos(2.0 * M_PI * f * s));
    }
}

/* Coefficient c(s,t) of -div(c grad u) = 0. */
double oracle_coef(int family, int coef_mode, const double* p, double s, double t)
{
    double w, ws, wt;
    density_w(family, p, s, t, &w, &ws, &wt);
    return coef_mode == 0 ? w : 1.0 / w;
}

/* Drift b = grad ln c = +-grad(w)/w (eq. ...Expanded). */
void oracle_drift(int family, int coef_mode, const double* p, double s, double t,
                  double b[2])
{
    double w, ws, wt;
    density_w(family, p, s, t, &w, &ws, &wt);
    double sign = coef_mode == 0 ? 1.0 : -1.0;
    if (family == 3) {                       /* grad ln w = grad L directly */
        double L, Ls, Lt;
        table_L(p, s, t, &L, &Ls, &Lt);
        b[0] = sign * Ls;
        b[1] = sign * Lt;
        return;
    }
    b[0] = sign * ws / w;
    b[1] = sign * wt / w;
}

/* ------------------------------------------------------- boundary lookup -- */
/* Linear interpolation of a table of n values at nodes tau_j = j/(n-1). */
double oracle_lookup(const double* T, int n, double tau)
{
    double x = tau * (double)(n - 1);
    int j = (int)floor(x);
    if (j > n - 2) j = n - 2;
    if (j < 0) j = 0;
    double frac = x - (double)j;
    return T[j] + frac * (T[j + 1] - T[j]);
}

/* Edge numbering of the boundary tables edges[comp][edge][n]:
 *   0 bottom (t=0, tangential s), 1 top (t=1, tangential s),
 *   2 left (s=0, tangential t),   3 right (s=1, tangential t). */
static double score(const double* edges, int n, int comp, int edge, double tau)
{
    return oracle_lookup(edges + ((size_t)comp * 4 + (size_t)edge) * (size_t)n, n, tau);
}

/* Exit test for the step x -> y.  Returns the edge crossed (0..3) or -1 if y is
 * inside the open square.  Sides are closed (a point on a side has exited).
 * The exit point is the intersection of the segment with the crossed side: for
 * each violated side theta = (x_d - side)/(x_d - y_d); the smallest theta wins,
 * an exact tie going to the s-sides.  The tangential coordinate is clamped to
 * [0,1]; the normal coordinate is the side value. */
int oracle_exit_point(double xs, double xt, double ys, double yt, double e[2])
{
    int side_s = -1, side_t = -1;
    double th_s = 2.0, th_t = 2.0;
    if (ys <= 0.0) { side_s = 2; th_s = (xs - 0.0) / (xs - ys); }
    else if (ys >= 1.0) { side_s = 3; th_s = (xs - 1.0) / (xs - ys); }
    if (yt <= 0.0) { side_t = 0; th_t = (xt - 0.0) / (xt - yt); }
    else if (yt >= 1.0) { side_t = 1; th_t = (xt - 1.0) / (xt - yt); }
    if (side_s < 0 && side_t < 0) return -1;
    int use_s = side_s >= 0 && (side_t < 0 || th_s <= th_t);
    if (use_s) {
        double tt = xt + th_s * (yt - xt);
        if (tt < 0.0) tt = 0.0;
        if (tt > 1.0) tt = 1.0;
        e[0] = side_s == 2 ? 0.0 : 1.0;
        e[1] = tt;
        return side_s;
    } else {
        double ss = xs + th_t * (ys - xs);
        if (ss < 0.0) ss = 0.0;
        if (ss > 1.0) ss = 1.0;
        e[0] = ss;
        e[1] = side_t == 0 ? 0.0 : 1.0;
        return side_t;
    }
}

/* Projection of an interior point on its nearest side (first minimum in the
 * order s=0, s=1, t=0, t=1); used for paths stopped by the step cap. */
static int nearest_side(double s, double t, double e[2])
{
    double d[4] = {s, 1.0 - s, t, 1.0 - t};
    int best = 0;
    for (int m = 1; m < 4; ++m)
        if (d[m] < d[best]) best = m;
    static const int edge_of[4] = {2, 3, 0, 1};
    e[0] = s; e[1] = t;
    if (best == 0) e[0] = 0.0;
    if (best == 1) e[0] = 1.0;
    if (best == 2) e[1] = 0.0;
    if (best == 3) e[1] = 1.0;
    return edge_of[best];
}

/* ------------------------------------------------------- Brownian bridge -- */
/* Brownian-bridge exit test (§2.2, after Gobet): given the end points x, y of
 * an Euler-Maruyama step that stayed inside, the process sqrt(2) W pinned at x
 * and y crossed the side s during the step with probability
 *   p_s = exp(-2 d_s(x) d_s(y) / (sigma^2 dt)) = exp(-d_s(x) d_s(y) / dt),
 * d_s = distance to side s (half-space approximation of the square).  Sides in
 * the order s=0, s=1, t=0, t=1 draw the uniforms U_m = (r_m + 1/2) 2^-32 of
 * Philox(counter = (k, path, node, 1)), k = index of the step; the first side
 * with U_m < p_m is crossed.  When d_s(x) d_s(y) >= 23 dt for every side no
 * crossing is possible (p < 2^-33 <= U), so no uniforms are drawn.  The exit
 * point is the side value with the mean of the two tangential coordinates.
 * Returns the edge crossed or -1; *tie = 1 if some |U - p| < 1e-12. */
int oracle_bridge_exit(double xs, double xt, double ys, double yt, double dt, uint64_t seed,
                       uint32_t node, uint32_t path, uint32_t k, double e[2], int* tie)
{
    double q[4] = {xs * ys, (1.0 - xs) * (1.0 - ys), xt * yt, (1.0 - xt) * (1.0 - yt)};
    int any = 0;
    for (int m = 0; m < 4; ++m)
        if (q[m] < 23.0 * dt) any = 1;
    if (!any) return -1;
    uint32_t ctr[4] = {k, path, node, 1u};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t r[4];
    oracle_philox4x32_10(ctr, key, r);
    static const int edge_of[4] = {2, 3, 0, 1};
    for (int m = 0; m < 4; ++m) {
        if (!(q[m] < 23.0 * dt)) continue;
        double p = exp(-q[m] / dt);
        double u = ((double)r[m] + 0.5) * 0x1p-32;
        if (fabs(u - p) < 1e-12) *tie = 1;
        if (u < p) {
            double ts = 0.5 * (xs + ys), tt = 0.5 * (xt + yt);
            if (ts < 0.0) ts = 0.0;
            if (ts > 1.0) ts = 1.0;
            if (tt < 0.0) tt = 0.0;
            if (tt > 1.0) tt = 1.0;
            e[0] = ts; e[1] = tt;
            if (m == 0) e[0] = 0.0;
            if (m == 1) e[0] = 1.0;
            if (m == 2) e[1] = 0.0;
            if (m == 3) e[1] = 1.0;
            return edge_of[m];
        }
    }
    return -1;
}

/* -------------------------------------------------------------- one path -- */
/* Runs path `path` from (s0,t0).  Returns the score F = (f, g) at the exit
 * point; *steps = Euler-Maruyama updates performed; *tie = 1 if any post-step
 * coordinate came within tie_delta of 0 or 1 (an exit decision that rounding
 * could flip); *capped = 1 if max_steps was reached without an exit.
 * stepper 0: constant step dt; 1: exponential time stepping with mean step
 * dt (lambda = 1/dt). */
void oracle_path(int n, double s0, double t0, uint32_t node, uint32_t path,
                 const double* edges, int family, int coef_mode, const double* p,
                 uint64_t seed, double dt, uint64_t max_steps, double tie_delta, int exit_test,
                 int stepper, double F[2], uint64_t* steps, int* tie, int* capped)
{
    double xs = s0, xt = t0;
    double z[4];
    double E[4] = {1.0, 1.0, 1.0, 1.0};
    int flag = 0;
    uint64_t k = 0;
    double e[2];
    int edge = -1;
    while (k < max_steps) {
        if ((k & 1u) == 0)
            oracle_normals(seed, node, path, (uint32_t)(k >> 1), z);
        if (stepper == 1 && (k & 3u) == 0)
            oracle_step_lengths(seed, node, path, (uint32_t)(k >> 2), E);
        const double* zk = z + 2 * (int)(k & 1u);
        double h = stepper == 1 ? dt * E[k & 3u] : dt;
        double sq = sqrt(2.0 * h);
        double b[2];
        oracle_drift(family, coef_mode, p, xs, xt, b);
        double ys = xs + b[0] * h + sq * zk[0];
        double yt = xt + b[1] * h + sq * zk[1];
        k += 1;
        if (fabs(ys) < tie_delta || fabs(ys - 1.0) < tie_delta ||
            fabs(yt) < tie_delta || fabs(yt - 1.0) < tie_delta)
            flag = 1;
        edge = oracle_exit_point(xs, xt, ys, yt, e);
        if (edge >= 0) break;
        if (exit_test == 1) {
            edge = oracle_bridge_exit(xs, xt, ys, yt, h, seed, node, path, (uint32_t)(k - 1), e,
                                      &flag);
            if (edge >= 0) break;
        }
        xs = ys;
        xt = yt;
    }
    *capped = 0;
    if (edge < 0) {
        edge = nearest_side(xs, xt, e);
        *capped = 1;
    }
    double tau = (edge <= 1) ? e[0] : e[1];
    F[0] = score(edges, n, 0, edge, tau);
    F[1] = score(edges, n, 1, edge, tau);
    *steps = k;
    *tie = flag;
}

/* ------------------------------------------------------------- one node -- */
/* Paths [path_begin, path_end) of node (i,j), node id `node` in the counter.
 * sums = {S_all[2], Q_all[2], S_nt[2], Q_nt[2]}: sums of d = F - X0 and d^2
 * over all paths and over paths not flagged as ties (plain sequential FP64).
 * counts = {paths, ties, non_exits, steps}. */
void oracle_mc_node(int n, int i, int j, uint32_t node, const double* edges,
                    int family, int coef_mode, const double* p, uint64_t seed,
                    uint64_t path_begin, uint64_t path_end, double dt,
                    uint64_t max_steps, double tie_delta, int exit_test, int stepper,
                    double sums[8], uint64_t counts[4])
{
    double s0 = (double)i / (double)(n - 1);
    double t0 = (double)j / (double)(n - 1);
    double x0[2] = {s0, t0};
    memset(sums, 0, 8 * sizeof(double));
    memset(counts, 0, 4 * sizeof(uint64_t));
    for (uint64_t q = path_begin; q < path_end; ++q) {
        double F[2];
        uint64_t st;
        int tie, capped;
        oracle_path(n, s0, t0, node, (uint32_t)q, edges, family, coef_mode, p, seed,
                    dt, max_steps, tie_delta, exit_test, stepper, F, &st, &tie, &capped);
        for (int c = 0; c < 2; ++c) {
            double d = F[c] - x0[c];
            sums[0 + c] += d;
            sums[2 + c] += d * d;
            if (!tie) {
                sums[4 + c] += d;
                sums[6 + c] += d * d;
            }
        }
        counts[0] += 1;
        counts[1] += (uint64_t)tie;
        counts[2] += (uint64_t)capped;
        counts[3] += st;
    }
}

/* c(s,t) on an array of points (used to assemble the finite-difference
 * operator and the 1D boundary forms without a call per point). */
void oracle_coef_array(int family, int coef_mode, const double* p, int64_t npts,
                       const double* s, const double* t, double* out)
{
    for (int64_t m = 0; m < npts; ++m)
        out[m] = oracle_coef(family, coef_mode, p, s[m], t[m]);
}
