// Subdomain solves of the SDD mesh generator (Bihlo & Haynes, §2.1, Fig. 1;
// §3.5): the interface Monte Carlo values and the boundary map are Dirichlet
// data, and every subdomain's conservative five-point system
//     sum_nbr c_edge (u_nbr - u_ij) = 0,   c at edge midpoints  (§3.2)
// is solved independently, once (no iteration between subdomains).
//
// One CTA (1024 threads) per subdomain, all subdomains of all meshes in one
// launch, largest subdomains first (they set the end of the launch).  The mesh
// u is FP64 [n][n][2] (the two components share the operator and are solved
// together, interleaved as double2).  Two solvers:
//   * red-black SOR in FP64;
//   * FP32 CG for the correction A d = r, wrapped in FP64 iterative
//     refinement (FP64 residual r = b - A u, u += d), preconditioned by a
//     geometric multigrid V-cycle (Galerkin coarse operators) or by the
//     diagonal (Jacobi).
// Each CTA iterates to its relative residual ||b - A u||_2 / ||b||_2 <= tol,
// stagnation or the iteration cap; the loops are bounded, never spin.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <utility>

#include "sdd_internal.h"
#include "mg.cuh"

namespace sdd {
namespace {

// CTA sizes a solve can be launched with (SolveArgs::threads); 1024 is the
// default, smaller CTAs suit small subdomains (more CTAs per SM).
constexpr int SOLVE_THREADS_DEFAULT = 1024;

// ------------------------------------------------------ coefficients ----
// Bilinear interpolant of a table of ln w at (s,t) (TABLE family): the cell
// holding (s,t), the last one on the upper sides.
__device__ double table_ln_w(const double* __restrict__ T, int tn, double s, double t)
{
    const double m = (double)(tn - 1);
    const double x = s * m, y = t * m;
    const int a = min(max((int)floor(x), 0), tn - 2), b = min(max((int)floor(y), 0), tn - 2);
    const double fa = x - (double)a, fb = y - (double)b;
    const double L00 = __ldg(T + b * tn + a), L10 = __ldg(T + b * tn + a + 1);
    const double L01 = __ldg(T + (b + 1) * tn + a), L11 = __ldg(T + (b + 1) * tn + a + 1);
    return (1.0 - fb) * ((1.0 - fa) * L00 + fa * L10) + fb * ((1.0 - fa) * L01 + fa * L11);
}

// c(s,t) = w or 1/w for the density families, FP64 (tab, tn: the TABLE
// family's device table).
__device__ double coef64(int family, int coef_mode, const double* __restrict__ p,
                         const double* __restrict__ tab, int tn, double s, double t)
{
    double w;
    if (family == SDD_FAMILY_TABLE) {
        w = exp(table_ln_w(tab, tn, s, t));
    } else if (family == SDD_FAMILY_RING) {
        const double ds = s - p[1], dtt = t - p[2];
        const double u = p[3] * (sqrt(ds * ds + dtt * dtt) - p[4]);
        const double e = exp(-2.0 * fabs(u));
        const double ope = 1.0 + e;
        w = 1.0 + p[0] * 4.0 * e / (ope * ope);           // A sech^2(u)
    } else if (family == SDD_FAMILY_RIDGE) {
        double sn, cn;
        sincospi(2.0 * p[4] * s, &sn, &cn);
        const double v = t - p[2] - p[3] * sn;
        w = 1.0 + p[0] * exp(-p[1] * v * v);
    } else {
        const int nb = (int)p[0];
        w = 1.0;
        for (int b = 0; b < nb; ++b) {
            const double* q = p + 1 + 5 * b;
            const double ds = s - q[1], dtt = t - q[2];
            w += q[0] * exp(-(q[3] * ds * ds + q[4] * dtt * dtt));
        }
    }
    return coef_mode == SDD_COEF_INV_W ? 1.0 / w : w;
}

struct CoefArgs {
    int n, family, coef_mode, tn;
    double p[SDD_MAX_PARAMS];
    const double* tab;
};

// cx[j][i] = c((i+1/2)h, jh), i < n-1;  cy[j][i] = c(ih, (j+1/2)h), j < n-1.
__global__ void k_edge_coefs(CoefArgs a, double* __restrict__ cx, double* __restrict__ cy,
                             float* __restrict__ cxf, float* __restrict__ cyf)
{
    const int n = a.n;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t m = (int64_t)n * (n - 1);
    if (g >= 2 * m) return;
    const double h = 1.0 / (double)(n - 1);
    if (g < m) {
        const int j = (int)(g / (n - 1)), i = (int)(g % (n - 1));
        const double c = coef64(a.family, a.coef_mode, a.p, a.tab, a.tn, ((double)i + 0.5) * h,
                                (double)j / (double)(n - 1));
        cx[g] = c;
        cxf[g] = (float)c;
    } else {
        const int64_t q = g - m;
        const int j = (int)(q / n), i = (int)(q % n);
        const double c = coef64(a.family, a.coef_mode, a.p, a.tab, a.tn, (double)i / (double)(n - 1),
                                ((double)j + 0.5) * h);
        cy[q] = c;
        cyf[q] = (float)c;
    }
}

// Boundary rows/columns from the tables (rows t=0 and t=1 include corners),
// then the interface values.
__global__ void k_fill_ring(int n, const double* __restrict__ edges, const int2* __restrict__ nodes,
                            int64_t n_nodes, const double* __restrict__ iface,
                            double2* __restrict__ u)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nb = 4 * (int64_t)n;
    if (g < nb) {
        const int e = (int)(g / n), k = (int)(g % n);
        const double v0 = edges[(0 * 4 + e) * (int64_t)n + k];
        const double v1 = edges[(1 * 4 + e) * (int64_t)n + k];
        int64_t idx;
        if (e == 0) idx = k;                                   // bottom, t = 0
        else if (e == 1) idx = (int64_t)(n - 1) * n + k;       // top, t = 1
        else {
            if (k == 0 || k == n - 1) return;                  // corners from the rows
            idx = (int64_t)k * n + (e == 2 ? 0 : n - 1);
        }
        u[idx] = make_double2(v0, v1);
    } else if (g - nb < n_nodes) {
        const int64_t v = g - nb;
        const int2 ij = nodes[v];
        u[(int64_t)ij.y * n + ij.x] = make_double2(iface[2 * v], iface[2 * v + 1]);
    }
}

// Batched form: one thread per boundary-table entry or interface node of any
// mesh of the batch (mesh found by binary search of the prefix offsets).
__global__ void k_fill_ring_batched(const FillDev* __restrict__ fill, const uint64_t* __restrict__ off,
                                    int n_meshes, uint64_t total)
{
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    int lo = 0, hi = n_meshes;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= g) lo = mid; else hi = mid;
    }
    const FillDev& F = fill[lo];
    const int64_t x = (int64_t)(g - off[lo]);
    const int n = F.n;
    double2* __restrict__ u = reinterpret_cast<double2*>(F.u);
    const int64_t nb = 4 * (int64_t)n;
    if (x < nb) {
        const int e = (int)(x / n), k = (int)(x % n);
        const double v0 = F.edges[(0 * 4 + e) * (int64_t)n + k];
        const double v1 = F.edges[(1 * 4 + e) * (int64_t)n + k];
        int64_t idx;
        if (e == 0) idx = k;
        else if (e == 1) idx = (int64_t)(n - 1) * n + k;
        else {
            if (k == 0 || k == n - 1) return;
            idx = (int64_t)k * n + (e == 2 ? 0 : n - 1);
        }
        u[idx] = make_double2(v0, v1);
    } else if (x - nb < F.n_nodes) {
        const int64_t v = x - nb;
        const int2 ij = F.nodes[v];
        u[(int64_t)ij.y * n + ij.x] = make_double2(F.iface[2 * v], F.iface[2 * v + 1]);
    }
}

// Transfinite (Coons) interpolation of each subdomain's ring as the start
// value of its interior.
__global__ void k_coons(SolveArgs a)
{
    const SubDev sd = a.subs[blockIdx.x];
    const SolveMeshDev& M = a.meshes ? a.meshes[sd.mesh] : a.single;
    const int n = M.n;
    double2* __restrict__ u = reinterpret_cast<double2*>(M.u);
    const int nx = sd.i1 - sd.i0 - 1, ny = sd.j1 - sd.j0 - 1;
    if (nx <= 0 || ny <= 0) return;
    const double2 c00 = u[(int64_t)sd.j0 * n + sd.i0], c10 = u[(int64_t)sd.j0 * n + sd.i1];
    const double2 c01 = u[(int64_t)sd.j1 * n + sd.i0], c11 = u[(int64_t)sd.j1 * n + sd.i1];
    const double wi = 1.0 / (double)(sd.i1 - sd.i0), wj = 1.0 / (double)(sd.j1 - sd.j0);
    for (int t = threadIdx.x; t < nx * ny; t += blockDim.x) {
        const int i = sd.i0 + 1 + t % nx, j = sd.j0 + 1 + t / nx;
        const double a = (double)(i - sd.i0) * wi, b = (double)(j - sd.j0) * wj;
        const double2 L = u[(int64_t)j * n + sd.i0], Rr = u[(int64_t)j * n + sd.i1];
        const double2 B = u[(int64_t)sd.j0 * n + i], T = u[(int64_t)sd.j1 * n + i];
        double2 v;
        v.x = (1 - a) * L.x + a * Rr.x + (1 - b) * B.x + b * T.x -
              ((1 - a) * (1 - b) * c00.x + a * (1 - b) * c10.x + (1 - a) * b * c01.x + a * b * c11.x);
        v.y = (1 - a) * L.y + a * Rr.y + (1 - b) * B.y + b * T.y -
              ((1 - a) * (1 - b) * c00.y + a * (1 - b) * c10.y + (1 - a) * b * c01.y + a * b * c11.y);
        u[(int64_t)j * n + i] = v;
    }
}

// --------------------------------------------------- block reductions ----
template <typename T, int K>
__device__ void block_sum(T (&v)[K], T* scratch /* >= K * 32 */)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < K; ++q)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
    __syncthreads();                       // scratch may still be read by a previous call
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < K; ++q) scratch[q * 32 + warp] = v[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < K; ++q) {
        T s = T(0);
        for (int w = 0; w < nw; ++w) s += scratch[q * 32 + w];   // fixed order
        v[q] = s;
    }
}

struct Box {
    int n, i0, i1, j0, j1, nx, ny;
    __device__ Box(const SubDev& sd, int n_) : n(n_), i0(sd.i0), i1(sd.i1), j0(sd.j0), j1(sd.j1)
    {
        nx = i1 - i0 - 1;
        ny = j1 - j0 - 1;
    }
};

// FP64 residual  r_ij = sum_nbr c (u_nbr - u_ij)  (= (b - A u)_ij) at node (i,j).
__device__ __forceinline__ double2 residual64(const SolveMeshDev& M, const double2* __restrict__ u,
                                              int n, int i, int j)
{
    const int64_t id = (int64_t)j * n + i;
    const double cE = M.cx[(int64_t)j * (n - 1) + i], cW = M.cx[(int64_t)j * (n - 1) + i - 1];
    const double cN = M.cy[id], cS = M.cy[id - n];
    const double2 c = u[id], e = u[id + 1], w = u[id - 1], nn = u[id + n], s = u[id - n];
    double2 r;
    r.x = cE * (e.x - c.x) + cW * (w.x - c.x) + cN * (nn.x - c.x) + cS * (s.x - c.x);
    r.y = cE * (e.y - c.y) + cW * (w.y - c.y) + cN * (nn.y - c.y) + cS * (s.y - c.y);
    return r;
}

// ||b||^2: b_ij = sum of c u_nbr over the Dirichlet (ring) neighbours.
__device__ double rhs_norm2(const SolveMeshDev& M, const Box& B, double* scratch)
{
    const int n = B.n;
    const double2* __restrict__ u = reinterpret_cast<const double2*>(M.u);
    double acc[1] = {0.0};
    for (int t = threadIdx.x; t < B.nx * B.ny; t += blockDim.x) {
        const int i = B.i0 + 1 + t % B.nx, j = B.j0 + 1 + t / B.nx;
        const bool w = i == B.i0 + 1, e = i == B.i1 - 1, s = j == B.j0 + 1, nn = j == B.j1 - 1;
        if (!(w | e | s | nn)) continue;
        const int64_t id = (int64_t)j * n + i;
        double bx = 0.0, by = 0.0;
        if (e) {
            const double c = M.cx[(int64_t)j * (n - 1) + i];
            const double2 v = u[id + 1];
            bx += c * v.x; by += c * v.y;
        }
        if (w) {
            const double c = M.cx[(int64_t)j * (n - 1) + i - 1];
            const double2 v = u[id - 1];
            bx += c * v.x; by += c * v.y;
        }
        if (nn) {
            const double c = M.cy[id];
            const double2 v = u[id + n];
            bx += c * v.x; by += c * v.y;
        }
        if (s) {
            const double c = M.cy[id - n];
            const double2 v = u[id - n];
            bx += c * v.x; by += c * v.y;
        }
        acc[0] += bx * bx + by * by;
    }
    block_sum<double, 1>(acc, scratch);
    return acc[0];
}

__device__ double residual_norm2(const SolveMeshDev& M, const Box& B, double* scratch)
{
    const double2* __restrict__ u = reinterpret_cast<const double2*>(M.u);
    double acc[1] = {0.0};
    for (int t = threadIdx.x; t < B.nx * B.ny; t += blockDim.x) {
        const int i = B.i0 + 1 + t % B.nx, j = B.j0 + 1 + t / B.nx;
        const double2 r = residual64(M, u, B.n, i, j);
        acc[0] += r.x * r.x + r.y * r.y;
    }
    block_sum<double, 1>(acc, scratch);
    return acc[0];
}

// ------------------------------------------------------------ SOR ----
__device__ void sor_box(const SolveMeshDev& M, const Box& B, SubStat& st, double* scratch)
{
    const int n = B.n;
    double2* __restrict__ u = reinterpret_cast<double2*>(M.u);
    double omega = M.omega;
    if (!(omega > 0.0 && omega < 2.0)) {
        const double rho = 0.5 * (cospi(1.0 / (B.nx + 1)) + cospi(1.0 / (B.ny + 1)));
        omega = 2.0 / (1.0 + sqrt(fmax(1.0 - rho * rho, 0.0)));
    }
    const double b2 = rhs_norm2(M, B, scratch);
    const double goal = M.tol * M.tol * fmax(b2, 1e-300);
    const int hx = (B.nx + 1) / 2;
    const int max_iter = M.max_iter;
    const int check = 8;
    double best = INFINITY;
    int stall = 0, it = 0;
    double r2 = residual_norm2(M, B, scratch);
    while (r2 > goal && it < max_iter) {
        for (int sweep = 0; sweep < check; ++sweep, ++it) {
#pragma unroll 1
            for (int color = 0; color < 2; ++color) {
                for (int t = threadIdx.x; t < B.ny * hx; t += blockDim.x) {
                    const int j = B.j0 + 1 + t / hx;
                    const int i = B.i0 + 1 + ((B.i0 + 1 + j + color) & 1) + 2 * (t % hx);
                    if (i >= B.i1) continue;
                    const int64_t id = (int64_t)j * n + i;
                    const double cE = M.cx[(int64_t)j * (n - 1) + i];
                    const double cW = M.cx[(int64_t)j * (n - 1) + i - 1];
                    const double cN = M.cy[id], cS = M.cy[id - n];
                    const double2 e = u[id + 1], w = u[id - 1], nn = u[id + n], s = u[id - n];
                    const double2 c = u[id];
                    const double dinv = 1.0 / (cE + cW + cN + cS);
                    const double gx = (cE * e.x + cW * w.x + cN * nn.x + cS * s.x) * dinv;
                    const double gy = (cE * e.y + cW * w.y + cN * nn.y + cS * s.y) * dinv;
                    u[id] = make_double2(c.x + omega * (gx - c.x), c.y + omega * (gy - c.y));
                }
                __syncthreads();
            }
        }
        r2 = residual_norm2(M, B, scratch);
        if (r2 < 0.98 * best) { best = r2; stall = 0; }
        else if (++stall >= 6) break;              // stagnated at rounding level
    }
    st.iterations = it;
    st.rel_residual = sqrt(r2 / fmax(b2, 1e-300));
    st.converged = r2 <= goal ? 1 : 0;
}

// ------------------------------------------- FP32 PCG + FP64 refinement ----
// FP32 CG preconditioned by the V-cycle, for the correction A d = r of each
// round of FP64 iterative refinement (u += d, r = b - A u in FP64).  Both
// components are solved together with their own step lengths.
__device__ void cg_mg_box(const SolveMeshDev& M, const Box& B, float* mg_base, SubStat& st,
                          double* scratch)
{
    __shared__ MgShape S;
    const int n = B.n;
    double2* __restrict__ u = reinterpret_cast<double2*>(M.u);
    const Work W = work_of(M);
    const float* __restrict__ cxf = M.cxf;
    const float* __restrict__ cyf = M.cyf;
    const int m = B.nx * B.ny;
    float* fs = reinterpret_cast<float*>(scratch);
    const Fine f{n, B.i0, B.j0, B.nx, B.ny, cxf, cyf};
    if (threadIdx.x == 0) mg_shape(B.nx, B.ny, S);

    // p = z = 0 on the ring: the SpMV and the smoothers read them there.
    for (int t = threadIdx.x; t < 2 * (B.nx + B.ny) + 4; t += blockDim.x) {
        int i, j;
        if (t < B.nx + 2) { i = B.i0 + t; j = B.j0; }
        else if (t < 2 * (B.nx + 2)) { i = B.i0 + (t - B.nx - 2); j = B.j1; }
        else if (t < 2 * (B.nx + 2) + B.ny) { i = B.i0; j = B.j0 + 1 + (t - 2 * (B.nx + 2)); }
        else { i = B.i1; j = B.j0 + 1 + (t - 2 * (B.nx + 2) - B.ny); }
        W.p[(int64_t)j * n + i] = make_float2(0.f, 0.f);
        W.z[(int64_t)j * n + i] = make_float2(0.f, 0.f);
    }
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
        const int i = B.i0 + 1 + t % B.nx, j = B.j0 + 1 + t / B.nx;
        const int64_t id = (int64_t)j * n + i;
        const float d = cxf[(int64_t)j * (n - 1) + i] + cxf[(int64_t)j * (n - 1) + i - 1] +
                        cyf[id] + cyf[id - n];
        W.dinv[id] = 1.0f / d;
    }
    __syncthreads();
    mg_setup(f, mg_base, S);
    const double b2 = rhs_norm2(M, B, scratch);
    const double goal = M.tol * M.tol * fmax(b2, 1e-300);
    const int max_inner = M.max_iter;
    const float inner_tol2 = 1e-10f;          // FP32 inner solve: ||r||_M / ||r0||_M <= 1e-5
    int total = 0;
    double r2 = 0.0, best = INFINITY;
    int rounds = 0, stall = 0;
    for (rounds = 0; rounds < 40; ++rounds) {
        // FP64 residual, cast to FP32; x = 0
        double acc[1] = {0.0};
        for (int t = threadIdx.x; t < m; t += blockDim.x) {
            const int i = B.i0 + 1 + t % B.nx, j = B.j0 + 1 + t / B.nx;
            const int64_t id = (int64_t)j * n + i;
            const double2 r = residual64(M, u, n, i, j);
            acc[0] += r.x * r.x + r.y * r.y;
            W.r[id] = make_float2((float)r.x, (float)r.y);
            W.x[id] = make_float2(0.f, 0.f);
        }
        block_sum<double, 1>(acc, scratch);
        r2 = acc[0];
        if (r2 <= goal) break;
        if (r2 < 0.5 * best) { best = r2; stall = 0; }
        else if (++stall >= 3) break;          // refinement no longer gains
        mg_vcycle(f, W, mg_base, S);           // z = M^-1 r
        float rz[2] = {0.f, 0.f};
        for (int t = threadIdx.x; t < m; t += blockDim.x) {
            const int64_t id = (int64_t)(B.j0 + 1 + t / B.nx) * n + (B.i0 + 1 + t % B.nx);
            const float2 r = W.r[id], z = W.z[id];
            W.p[id] = z;
            rz[0] += r.x * z.x;
            rz[1] += r.y * z.y;
        }
        block_sum<float, 2>(rz, fs + 64);
        const float rz0 = fmaxf(rz[0], rz[1]);
        float rzc[2] = {rz[0], rz[1]};
        int it = 0;
        for (; it < max_inner; ++it) {
            __syncthreads();                   // p complete before the SpMV
            float pq[2] = {0.f, 0.f};
            for (int t = threadIdx.x; t < m; t += blockDim.x) {
                const int i = B.i0 + 1 + t % B.nx, j = B.j0 + 1 + t / B.nx;
                const int64_t id = (int64_t)j * n + i;
                const float cE = cxf[(int64_t)j * (n - 1) + i], cW = cxf[(int64_t)j * (n - 1) + i - 1];
                const float cN = cyf[id], cS = cyf[id - n];
                const float2 c = W.p[id], e = W.p[id + 1], w = W.p[id - 1];
                const float2 nn = W.p[id + n], s = W.p[id - n];
                const float d = cE + cW + cN + cS;
                float2 q;
                q.x = d * c.x - (cE * e.x + cW * w.x + cN * nn.x + cS * s.x);
                q.y = d * c.y - (cE * e.y + cW * w.y + cN * nn.y + cS * s.y);
                W.q[id] = q;
                pq[0] += c.x * q.x;
                pq[1] += c.y * q.y;
            }
            block_sum<float, 2>(pq, fs);
            const float al0 = pq[0] > 0.f ? rzc[0] / pq[0] : 0.f;
            const float al1 = pq[1] > 0.f ? rzc[1] / pq[1] : 0.f;
            for (int t = threadIdx.x; t < m; t += blockDim.x) {
                const int64_t id = (int64_t)(B.j0 + 1 + t / B.nx) * n + (B.i0 + 1 + t % B.nx);
                const float2 p = W.p[id], q = W.q[id];
                float2 x = W.x[id], r = W.r[id];
                x.x += al0 * p.x; x.y += al1 * p.y;
                r.x -= al0 * q.x; r.y -= al1 * q.y;
                W.x[id] = x;
                W.r[id] = r;
            }
            __syncthreads();                   // r complete before the V-cycle
            mg_vcycle(f, W, mg_base, S);
            float nz[2] = {0.f, 0.f};
            for (int t = threadIdx.x; t < m; t += blockDim.x) {
                const int64_t id = (int64_t)(B.j0 + 1 + t / B.nx) * n + (B.i0 + 1 + t % B.nx);
                const float2 r = W.r[id], z = W.z[id];
                nz[0] += r.x * z.x;
                nz[1] += r.y * z.y;
            }
            block_sum<float, 2>(nz, fs + 64);
            const float be0 = rzc[0] > 0.f ? nz[0] / rzc[0] : 0.f;
            const float be1 = rzc[1] > 0.f ? nz[1] / rzc[1] : 0.f;
            rzc[0] = nz[0];
            rzc[1] = nz[1];
            for (int t = threadIdx.x; t < m; t += blockDim.x) {
                const int64_t id = (int64_t)(B.j0 + 1 + t / B.nx) * n + (B.i0 + 1 + t % B.nx);
                const float2 z = W.z[id], p = W.p[id];
                W.p[id] = make_float2(z.x + be0 * p.x, z.y + be1 * p.y);
            }
            if (fmaxf(rzc[0], rzc[1]) <= inner_tol2 * rz0) { ++it; break; }
        }
        total += it;
        __syncthreads();
        for (int t = threadIdx.x; t < m; t += blockDim.x) {
            const int i = B.i0 + 1 + t % B.nx, j = B.j0 + 1 + t / B.nx;
            const int64_t id = (int64_t)j * n + i;
            const float2 x = W.x[id];
            double2 v = u[id];
            v.x += (double)x.x;
            v.y += (double)x.y;
            u[id] = v;
        }
        __syncthreads();
    }
    st.iterations = total;
    st.rel_residual = sqrt(r2 / fmax(b2, 1e-300));
    st.converged = r2 <= goal ? 1 : 0;
}

__device__ void cg_box(const SolveMeshDev& M, const Box& B, SubStat& st, double* scratch)
{
    const int n = B.n;
    double2* __restrict__ u = reinterpret_cast<double2*>(M.u);
    const Work W = work_of(M);
    const float* __restrict__ cxf = M.cxf;
    const float* __restrict__ cyf = M.cyf;
    const int m = B.nx * B.ny;
    float* fs = reinterpret_cast<float*>(scratch);

    // p = 0 on the ring: the SpMV reads it at the interior's neighbours.
    for (int t = threadIdx.x; t < 2 * (B.nx + B.ny) + 4; t += blockDim.x) {
        int i, j;
        if (t < B.nx + 2) { i = B.i0 + t; j = B.j0; }
        else if (t < 2 * (B.nx + 2)) { i = B.i0 + (t - B.nx - 2); j = B.j1; }
        else if (t < 2 * (B.nx + 2) + B.ny) { i = B.i0; j = B.j0 + 1 + (t - 2 * (B.nx + 2)); }
        else { i = B.i1; j = B.j0 + 1 + (t - 2 * (B.nx + 2) - B.ny); }
        W.p[(int64_t)j * n + i] = make_float2(0.f, 0.f);
    }
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
        const int i = B.i0 + 1 + t % B.nx, j = B.j0 + 1 + t / B.nx;
        const int64_t id = (int64_t)j * n + i;
        const float d = cxf[(int64_t)j * (n - 1) + i] + cxf[(int64_t)j * (n - 1) + i - 1] +
                        cyf[id] + cyf[id - n];
        W.dinv[id] = 1.0f / d;
    }
    const double b2 = rhs_norm2(M, B, scratch);
    const double goal = M.tol * M.tol * fmax(b2, 1e-300);
    const int max_inner = M.max_iter;
    const float inner_tol2 = 1e-10f;          // FP32 inner solve: ||r|| / ||r0|| <= 1e-5
    int total = 0;
    double r2 = 0.0, best = INFINITY;
    int rounds = 0, stall = 0;
    for (rounds = 0; rounds < 40; ++rounds) {
        // FP64 residual, cast to FP32; x = 0; p = z = D^-1 r
        double acc[1] = {0.0};
        float rz[2] = {0.f, 0.f};
        for (int t = threadIdx.x; t < m; t += blockDim.x) {
            const int i = B.i0 + 1 + t % B.nx, j = B.j0 + 1 + t / B.nx;
            const int64_t id = (int64_t)j * n + i;
            const double2 r = residual64(M, u, n, i, j);
            acc[0] += r.x * r.x + r.y * r.y;
            const float2 rf = make_float2((float)r.x, (float)r.y);
            const float di = W.dinv[id];
            const float2 z = make_float2(rf.x * di, rf.y * di);
            W.r[id] = rf;
            W.p[id] = z;
            W.x[id] = make_float2(0.f, 0.f);
            rz[0] += rf.x * z.x;
            rz[1] += rf.y * z.y;
        }
        block_sum<double, 1>(acc, scratch);
        r2 = acc[0];
        if (r2 <= goal) break;
        if (r2 < 0.5 * best) { best = r2; stall = 0; }
        else if (++stall >= 3) break;          // refinement no longer gains
        block_sum<float, 2>(rz, fs + 64);
        const float rz0 = fmaxf(rz[0], rz[1]);
        float rzc[2] = {rz[0], rz[1]};
        int it = 0;
        for (; it < max_inner; ++it) {
            __syncthreads();                   // p complete before the SpMV
            float pq[2] = {0.f, 0.f};
            for (int t = threadIdx.x; t < m; t += blockDim.x) {
                const int i = B.i0 + 1 + t % B.nx, j = B.j0 + 1 + t / B.nx;
                const int64_t id = (int64_t)j * n + i;
                const float cE = cxf[(int64_t)j * (n - 1) + i], cW = cxf[(int64_t)j * (n - 1) + i - 1];
                const float cN = cyf[id], cS = cyf[id - n];
                const float2 c = W.p[id], e = W.p[id + 1], w = W.p[id - 1];
                const float2 nn = W.p[id + n], s = W.p[id - n];
                const float d = cE + cW + cN + cS;
                float2 q;
                q.x = d * c.x - (cE * e.x + cW * w.x + cN * nn.x + cS * s.x);
                q.y = d * c.y - (cE * e.y + cW * w.y + cN * nn.y + cS * s.y);
                W.q[id] = q;
                pq[0] += c.x * q.x;
                pq[1] += c.y * q.y;
            }
            block_sum<float, 2>(pq, fs);
            const float al0 = pq[0] > 0.f ? rzc[0] / pq[0] : 0.f;
            const float al1 = pq[1] > 0.f ? rzc[1] / pq[1] : 0.f;
            float nz[2] = {0.f, 0.f};
            for (int t = threadIdx.x; t < m; t += blockDim.x) {
                const int i = B.i0 + 1 + t % B.nx, j = B.j0 + 1 + t / B.nx;
                const int64_t id = (int64_t)j * n + i;
                const float2 p = W.p[id], q = W.q[id];
                float2 x = W.x[id], r = W.r[id];
                x.x += al0 * p.x; x.y += al1 * p.y;
                r.x -= al0 * q.x; r.y -= al1 * q.y;
                W.x[id] = x;
                W.r[id] = r;
                const float di = W.dinv[id];
                nz[0] += r.x * r.x * di;
                nz[1] += r.y * r.y * di;
            }
            block_sum<float, 2>(nz, fs + 64);
            const float be0 = rzc[0] > 0.f ? nz[0] / rzc[0] : 0.f;
            const float be1 = rzc[1] > 0.f ? nz[1] / rzc[1] : 0.f;
            rzc[0] = nz[0];
            rzc[1] = nz[1];
            for (int t = threadIdx.x; t < m; t += blockDim.x) {
                const int i = B.i0 + 1 + t % B.nx, j = B.j0 + 1 + t / B.nx;
                const int64_t id = (int64_t)j * n + i;
                const float di = W.dinv[id];
                const float2 r = W.r[id], p = W.p[id];
                W.p[id] = make_float2(r.x * di + be0 * p.x, r.y * di + be1 * p.y);
            }
            if (fmaxf(rzc[0], rzc[1]) <= inner_tol2 * rz0) { ++it; break; }
        }
        total += it;
        __syncthreads();
        for (int t = threadIdx.x; t < m; t += blockDim.x) {
            const int i = B.i0 + 1 + t % B.nx, j = B.j0 + 1 + t / B.nx;
            const int64_t id = (int64_t)j * n + i;
            const float2 x = W.x[id];
            double2 v = u[id];
            v.x += (double)x.x;
            v.y += (double)x.y;
            u[id] = v;
        }
        __syncthreads();
    }
    st.iterations = total;
    st.rel_residual = sqrt(r2 / fmax(b2, 1e-300));
    st.converged = r2 <= goal ? 1 : 0;
}

// MASK: solvers compiled into the kernel (bit 0 SOR, bit 1 multigrid CG, bit
// 2 Jacobi CG), so a launch whose subdomains all use one solver gets a kernel
// with that solver only.  THREADS < 1024: register use capped so that
// 1024 / THREADS CTAs share an SM, whose barrier waits then overlap (a batch
// of many subdomains: two CTAs of 512 per SM solve config-3's 7000
// subdomains in 28 ms instead of 38 ms with one CTA of 1024).
template <int MASK, int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS)
k_solve(SolveArgs a)
{
    __shared__ double scratch[128];
    const SubDev sd = a.subs[blockIdx.x];
    const SolveMeshDev& M = a.meshes ? a.meshes[sd.mesh] : a.single;
    const Box B(sd, M.n);
    SubStat st;
    st.iterations = 0;
    st.converged = 1;
    st.rel_residual = 0.0;
    if (B.nx > 0 && B.ny > 0) {
        if constexpr (MASK == 2) cg_mg_box(M, B, M.mg + sd.mg_off, st, scratch);
        else if constexpr (MASK == 1) sor_box(M, B, st, scratch);
        else if constexpr (MASK == 4) cg_box(M, B, st, scratch);
        else {
            if (M.solver == SDD_SOLVER_CG_FP32_REFINE) cg_mg_box(M, B, M.mg + sd.mg_off, st, scratch);
            else if (M.solver == SDD_SOLVER_CG_JACOBI_FP32_REFINE) cg_box(M, B, st, scratch);
            else sor_box(M, B, st, scratch);
        }
    }
    if (threadIdx.x == 0) a.stats[sd.slot] = st;
}

// Mesh quality (§3.1, §3.3): per cell the Jacobian of (s,t) -> u from the
// mean of the cell's two edge differences per direction, Q = 1/2 |J|_F^2 /
// det J (folded when det J <= 0); per node |w(u) - w(ref)|.  Block
// reductions, then atomics (max of non-negative bit patterns, sums).
__device__ __forceinline__ bool cell_q(const double2* __restrict__ u, int n, int i, int j, double& q)
{
    const double h = 1.0 / (double)(n - 1);
    const double2 a00 = u[(int64_t)j * n + i], a10 = u[(int64_t)j * n + i + 1];
    const double2 a01 = u[(int64_t)(j + 1) * n + i], a11 = u[(int64_t)(j + 1) * n + i + 1];
    const double xs = ((a10.x - a00.x) + (a11.x - a01.x)) / (2 * h);
    const double ys = ((a10.y - a00.y) + (a11.y - a01.y)) / (2 * h);
    const double xt = ((a01.x - a00.x) + (a11.x - a10.x)) / (2 * h);
    const double yt = ((a01.y - a00.y) + (a11.y - a10.y)) / (2 * h);
    const double det = xs * yt - xt * ys;
    if (!(det > 0.0)) return false;
    q = 0.5 * (xs * xs + xt * xt + ys * ys + yt * yt) / det;
    return true;
}

struct QualityArgs {
    int n, family, tn;
    double p[SDD_MAX_PARAMS];
    const double* tab;
};

__global__ void __launch_bounds__(256) k_quality(QualityArgs a, const double2* __restrict__ u,
                                                 const double2* __restrict__ ref,
                                                 QualityDev* __restrict__ out)
{
    __shared__ double scratch[128];
    const int n = a.n;
    const int64_t cells = (int64_t)(n - 1) * (n - 1);
    const int64_t nodes = (int64_t)n * n;
    double qmax[2] = {0.0, 0.0}, qsum[2] = {0.0, 0.0}, linf = 0.0;
    unsigned long long folds[2] = {0ull, 0ull};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nodes; g += stride) {
        const int i = (int)(g % n), j = (int)(g / n);
        if (g < nodes && i < n - 1 && j < n - 1) {
            double q;
            if (cell_q(u, n, i, j, q)) { qmax[0] = fmax(qmax[0], q); qsum[0] += q; } else ++folds[0];
            if (ref) {
                if (cell_q(ref, n, i, j, q)) { qmax[1] = fmax(qmax[1], q); qsum[1] += q; } else ++folds[1];
            }
        }
        if (ref) {
            const double2 x = u[g], y = ref[g];
            linf = fmax(linf, fabs(coef64(a.family, SDD_COEF_W, a.p, a.tab, a.tn, x.x, x.y) -
                                   coef64(a.family, SDD_COEF_W, a.p, a.tab, a.tn, y.x, y.y)));
        }
    }
    (void)cells;
    double v[4] = {qsum[0], qsum[1], (double)folds[0], (double)folds[1]};
    block_sum<double, 4>(v, scratch);
    // maxima: warp then block by shuffles and shared memory
    double m[3] = {qmax[0], qmax[1], linf};
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) m[q] = fmax(m[q], __shfl_xor_sync(0xffffffffu, m[q], off));
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&out->q_max_bits, (unsigned long long)__double_as_longlong(m[0]));
        atomicMax(&out->q_ref_max_bits, (unsigned long long)__double_as_longlong(m[1]));
        atomicMax(&out->l_inf_bits, (unsigned long long)__double_as_longlong(m[2]));
    }
    if (threadIdx.x == 0) {
        atomicAdd(&out->q_sum, v[0]);
        atomicAdd(&out->q_ref_sum, v[1]);
        atomicAdd(&out->folds, (unsigned long long)v[2]);
        atomicAdd(&out->ref_folds, (unsigned long long)v[3]);
    }
}

// Perona-Malik smoothing (§3.4, eq. PeronaMalikDiffusion), one FTCS step
// u -> v per launch, both components: each of a node's four edges conducts
// with g = exp(-(d/h)^2 / k^2) of its own difference d = u_nb - u, so
//   v = u + r (g_E d_E + g_W d_W + g_N d_N + g_S d_S),  r = dt / h^2;
// boundary nodes are copied, and so are the nodes of held lines (hold[i]
// bit 0: column i, hold[j] bit 1: row j; hold may be null): with the
// subdomains' interface lines held, every subdomain is smoothed on its own
// (§3.5, §4).  One thread per node, mesh rows of double2.
__device__ __forceinline__ double pm_flux(double d, double h, double k2)
{
    const double t = d / h;
    return exp(-(t * t) / k2) * d;
}

__global__ void __launch_bounds__(256) k_pm_step(int n, const double2* __restrict__ u,
                                                 double2* __restrict__ v, double h, double r,
                                                 double k2, const uint8_t* __restrict__ hold)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (int64_t)n * n) return;
    const int i = (int)(g % n), j = (int)(g / n);
    const double2 c = u[g];
    if (i == 0 || j == 0 || i == n - 1 || j == n - 1 ||
        (hold && ((hold[i] & 1u) | (hold[j] & 2u)))) {
        v[g] = c;
        return;
    }
    const double2 E = u[g + 1], Wn = u[g - 1], N = u[g + n], S = u[g - n];
    double2 o;
    o.x = c.x + r * (pm_flux(E.x - c.x, h, k2) + pm_flux(Wn.x - c.x, h, k2) +
                     pm_flux(N.x - c.x, h, k2) + pm_flux(S.x - c.x, h, k2));
    o.y = c.y + r * (pm_flux(E.y - c.y, h, k2) + pm_flux(Wn.y - c.y, h, k2) +
                     pm_flux(N.y - c.y, h, k2) + pm_flux(S.y - c.y, h, k2));
    v[g] = o;
}

}  // namespace

int launch_quality(int n, int family, const double* params, const double* tab, int tn,
                   const double* u, const double* ref, QualityDev* d_out, cudaStream_t stream)
{
    QualityArgs a;
    a.n = n;
    a.family = family;
    a.tab = tab;
    a.tn = tn;
    for (int q = 0; q < SDD_MAX_PARAMS; ++q) a.p[q] = params[q];
    SDD_CUDA(cudaMemsetAsync(d_out, 0, sizeof(QualityDev), stream));
    const int64_t nodes = (int64_t)n * n;
    const unsigned blocks = (unsigned)std::min<int64_t>((nodes + 255) / 256, 4096);
    k_quality<<<blocks, 256, 0, stream>>>(a, reinterpret_cast<const double2*>(u),
                                          reinterpret_cast<const double2*>(ref), d_out);
    SDD_CUDA(cudaGetLastError());
    count_launch();
    return SDD_OK;
}

int launch_smooth(int n, double* u, double* scratch, int steps, double dt, double k,
                  const uint8_t* hold, cudaStream_t stream)
{
    if (steps <= 0) return SDD_OK;
    const double h = 1.0 / (double)(n - 1);
    const double r = dt / (h * h), k2 = k * k;
    const int64_t nodes = (int64_t)n * n;
    const unsigned blocks = (unsigned)((nodes + 255) / 256);
    double2* a = reinterpret_cast<double2*>(u);
    double2* b = reinterpret_cast<double2*>(scratch);
    for (int s = 0; s < steps; ++s) {
        k_pm_step<<<blocks, 256, 0, stream>>>(n, a, b, h, r, k2, hold);
        SDD_CUDA(cudaGetLastError());
        count_launch();
        std::swap(a, b);
    }
    if (a != reinterpret_cast<double2*>(u))          // odd step count: result in scratch
        SDD_CUDA(cudaMemcpyAsync(u, a, (size_t)nodes * sizeof(double2), cudaMemcpyDeviceToDevice,
                                 stream));
    return SDD_OK;
}

int launch_edge_coefs(int n, int family, int coef_mode, const double* params, const double* tab,
                      int tn, double* cx, double* cy, float* cxf, float* cyf, cudaStream_t stream)
{
    CoefArgs a;
    a.n = n;
    a.family = family;
    a.coef_mode = coef_mode;
    a.tab = tab;
    a.tn = tn;
    for (int q = 0; q < SDD_MAX_PARAMS; ++q) a.p[q] = params[q];
    const int64_t total = 2 * (int64_t)n * (n - 1);
    k_edge_coefs<<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(a, cx, cy, cxf, cyf);
    SDD_CUDA(cudaGetLastError());
    count_launch();
    return SDD_OK;
}

int launch_fill_mesh(int n, const double* edges, const int2* nodes, int64_t n_nodes,
                     const double* iface, double* u, const SubDev* subs, int n_subs,
                     cudaStream_t stream)
{
    (void)subs;
    (void)n_subs;
    const int64_t total = 4 * (int64_t)n + n_nodes;
    k_fill_ring<<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(
        n, edges, nodes, n_nodes, iface, reinterpret_cast<double2*>(u));
    SDD_CUDA(cudaGetLastError());
    count_launch();
    return SDD_OK;
}

int launch_fill_batched(const FillDev* d_fill, const uint64_t* d_off, int n_meshes,
                        uint64_t total, cudaStream_t stream)
{
    if (total == 0) return SDD_OK;
    k_fill_ring_batched<<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(d_fill, d_off,
                                                                             n_meshes, total);
    SDD_CUDA(cudaGetLastError());
    count_launch();
    return SDD_OK;
}

int launch_solve(const SolveArgs& args, cudaStream_t stream)
{
    if (args.n_subs <= 0) return SDD_OK;
    k_coons<<<args.n_subs, 256, 0, stream>>>(args);
    SDD_CUDA(cudaGetLastError());
    count_launch();
    const int t = args.threads == 256 || args.threads == 512 ? args.threads : SOLVE_THREADS_DEFAULT;
    // one solver in the launch: a kernel with that solver only; a mix: all three
    void (*k)(SolveArgs) = nullptr;
    const int sm = args.solver_mask;
    if (t == 256)
        k = sm == 1 ? k_solve<1, 256> : sm == 2 ? k_solve<2, 256> : sm == 4 ? k_solve<4, 256> : k_solve<7, 256>;
    else if (t == 512)
        k = sm == 1 ? k_solve<1, 512> : sm == 2 ? k_solve<2, 512> : sm == 4 ? k_solve<4, 512> : k_solve<7, 512>;
    else
        k = sm == 1 ? k_solve<1, 1024> : sm == 2 ? k_solve<2, 1024> : sm == 4 ? k_solve<4, 1024> : k_solve<7, 1024>;
    k<<<args.n_subs, t, 0, stream>>>(args);
    SDD_CUDA(cudaGetLastError());
    count_launch();
    return SDD_OK;
}

}  // namespace sdd
