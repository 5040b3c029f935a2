// Geometric multigrid for the subdomain solves (device functions, one CTA
// per subdomain): the CG workspace, the coarse levels, the Galerkin set-up,
// the smoothers, the transfers and the V-cycle.  Included by solve.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sdd_internal.h"

namespace sdd {
namespace {

// Workspace per grid node (floats): r(2) p(2) q(2) x(2) z(2) dinv(1).
struct Work {
    float2* r; float2* p; float2* q; float2* x; float2* z; float* dinv;
};

__device__ __forceinline__ Work work_of(const SolveMeshDev& M)
{
    const int64_t nn = (int64_t)M.n * M.n;
    Work w;
    w.r = reinterpret_cast<float2*>(M.work);
    w.p = w.r + nn;
    w.q = w.p + nn;
    w.x = w.q + nn;
    w.z = w.x + nn;
    w.dinv = reinterpret_cast<float*>(w.z + nn);
    return w;
}

// ------------------------------------------------------- multigrid ----
// Geometric multigrid V-cycle as the preconditioner of the FP32 CG: the
// interior of a subdomain (level 0, the conservative five-point operator of
// §3.2 with c at edge midpoints) and coarse levels of half the nodes per side
// (MgShape), with bilinear prolongation P, restriction P^T and the Galerkin
// operators A_{l+1} = P^T A_l P (nine-point stencils, computed in the kernel
// from the FP32 edge coefficients).  Smoothing: red-black Gauss-Seidel on
// level 0, four-colour Gauss-Seidel on the nine-point levels, colours in
// reverse order after the coarse correction, and a fixed number of damped
// Jacobi sweeps by one warp on the coarsest level: a fixed symmetric
// positive definite operator, so plain CG stays valid with it.  It only
// preconditions: the FP64 refinement and the CG's own residuals set the
// solution, so the fixed point is the one the five-point system defines.
struct MgLevel {
    int nx, ny, pitch, cx, cy, plane;
    float* a;                 // 9 stencil planes: a[k * plane + idx], k = (dy + 1) * 3 + dx + 1
    float2* x;
    float2* b;
    float2* t;
    __device__ __forceinline__ int idx(int I, int J) const { return J * pitch + I; }
};

__device__ __forceinline__ MgLevel mg_level(float* base, const MgShape& S, int l)
{
    MgLevel L;
    L.nx = S.nx[l];
    L.ny = S.ny[l];
    L.pitch = L.nx + 2;
    L.cx = S.cx[l];
    L.cy = S.cy[l];
    L.plane = S.plane[l];
    L.a = base + S.off[l];
    L.x = reinterpret_cast<float2*>(L.a + 9 * (int64_t)L.plane);
    L.b = L.x + L.plane;
    L.t = L.b + L.plane;
    return L;
}

// Bilinear interpolation weight of the fine offset d (per axis) to a coarse
// node: 1 at the node, 1/2 one fine step away, along a coarsened axis; along
// an axis kept as it is, 1 at the node only.
__device__ __forceinline__ float pw(int d, int coarsened)
{
    return d == 0 ? 1.f : (coarsened && (d == 1 || d == -1)) ? 0.5f : 0.f;
}

// (P x_C) at node (I, J) of the next finer level: the coarse nodes around
// it, weighted as pw(); the coarse x planes have a zero ring, which every
// index here stays inside.
__device__ __forceinline__ float2 mg_interp(const MgLevel& C, int I, int J)
{
    int i0 = I, i1 = I, j0 = J, j1 = J;
    float wi0 = 1.f, wi1 = 0.f, wj0 = 1.f, wj1 = 0.f;
    if (C.cx) {
        if (I & 1) { i0 = (I - 1) >> 1; i1 = (I + 1) >> 1; wi0 = wi1 = 0.5f; }
        else { i0 = i1 = I >> 1; }
    }
    if (C.cy) {
        if (J & 1) { j0 = (J - 1) >> 1; j1 = (J + 1) >> 1; wj0 = wj1 = 0.5f; }
        else { j0 = j1 = J >> 1; }
    }
    const float2 a = C.x[C.idx(i0, j0)], b = C.x[C.idx(i1, j0)];
    const float2 c = C.x[C.idx(i0, j1)], d = C.x[C.idx(i1, j1)];
    float2 v;
    v.x = wj0 * (wi0 * a.x + wi1 * b.x) + wj1 * (wi0 * c.x + wi1 * d.x);
    v.y = wj0 * (wi0 * a.y + wi1 * b.y) + wj1 * (wi0 * c.y + wi1 * d.y);
    return v;
}

// Level 0 viewed through subdomain-local indices (I, J) = (i - i0, j - j0),
// interior 1..nx, 1..ny.
struct Fine {
    int n, i0, j0, nx, ny;
    const float* cxf;
    const float* cyf;
    __device__ __forceinline__ int64_t id(int I, int J) const { return (int64_t)(j0 + J) * n + (i0 + I); }
    // five-point coefficients at (I, J): east, west, north, south
    __device__ __forceinline__ void c4(int I, int J, float& e, float& w, float& nn, float& s) const
    {
        const int64_t r = (int64_t)(j0 + J) * (n - 1) + (i0 + I);
        e = cxf[r];
        w = cxf[r - 1];
        const int64_t g = id(I, J);
        nn = cyf[g];
        s = cyf[g - n];
    }
};

// Galerkin stencil of coarse node (I, J) of level C from the finer level:
// sum over the fine nodes f of the node's hat function (weight w_f) and their
// stencil neighbours g (A_fg) of w_f A_fg P(g, J') for the coarse nodes J'
// around (I, J).  Fine: the five-point level 0 (FINE = true) or a nine-point
// level F.  CX, CY: whether C halves the x / y side of F.  Every offset is a
// compile-time constant once the loops are unrolled, so each term lands in a
// fixed entry of `out`, in the order f, g, J' (row by row); only the bounds
// (fine nodes and g inside the interior, J' a coarse interior node) are
// tested at run time.
template <bool FINE, int CX, int CY>
__device__ __forceinline__ void galerkin_node(const Fine& f0, const MgLevel& F, const MgLevel& C,
                                              int I, int J, float out[9])
{
#pragma unroll
    for (int k = 0; k < 9; ++k) out[k] = 0.f;
    const int fnx = FINE ? f0.nx : F.nx, fny = FINE ? f0.ny : F.ny;
    const int ci = CX ? 2 * I : I, cj = CY ? 2 * J : J;          // the node on the fine level
    bool cok[9];                                                 // coarse neighbour exists
#pragma unroll
    for (int d = 0; d < 9; ++d) {
        const int Ip = I + d % 3 - 1, Jp = J + d / 3 - 1;
        cok[d] = Ip >= 1 && Ip <= C.nx && Jp >= 1 && Jp <= C.ny;
    }
#pragma unroll
    for (int b = -1; b <= 1; ++b) {
        const float wb = pw(b, CY);
        if (wb == 0.f) continue;
        const int fj = cj + b;
#pragma unroll
        for (int a = -1; a <= 1; ++a) {
            const float wa = pw(a, CX);
            if (wa == 0.f) continue;
            const int fi = ci + a;
            if (fj < 1 || fj > fny || fi < 1 || fi > fnx) continue;
            const float wf = wa * wb;
            // the fine row of A at f: (gi, gj) offsets with value v
            float v[9];
            if constexpr (FINE) {
                float e, w, nn, s;
                f0.c4(fi, fj, e, w, nn, s);
                v[0] = 0.f; v[1] = -s; v[2] = 0.f;
                v[3] = -w; v[4] = e + w + nn + s; v[5] = -e;
                v[6] = 0.f; v[7] = -nn; v[8] = 0.f;
            } else {
                const int q = F.idx(fi, fj);
#pragma unroll
                for (int k = 0; k < 9; ++k) v[k] = F.a[k * F.plane + q];
            }
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                if (FINE && (k == 0 || k == 2 || k == 6 || k == 8)) continue;   // five points
                const int kx = k % 3 - 1, ky = k / 3 - 1;
                const int gi = fi + kx, gj = fj + ky;
                if (gi < 1 || gi > fnx || gj < 1 || gj > fny) continue;   // ring: no unknown
                const float fv = wf * v[k];
#pragma unroll
                for (int d = 0; d < 9; ++d) {
                    const int dI = d % 3 - 1, dJ = d / 3 - 1;
                    // offset of g from coarse node (I + dI, J + dJ) on the fine level
                    const int ox = CX ? a + kx - 2 * dI : a + kx - dI;
                    const int oy = CY ? b + ky - 2 * dJ : b + ky - dJ;
                    const float wx = pw(ox, CX), wy = pw(oy, CY);
                    if (wx == 0.f || wy == 0.f) continue;
                    if (cok[d]) out[d] += fv * wx * wy;
                }
            }
        }
    }
}

template <bool FINE>
__device__ __forceinline__ void galerkin_node_any(const Fine& f0, const MgLevel& F,
                                                  const MgLevel& C, int I, int J, float out[9])
{
    if (C.cx && C.cy) galerkin_node<FINE, 1, 1>(f0, F, C, I, J, out);
    else if (C.cx) galerkin_node<FINE, 1, 0>(f0, F, C, I, J, out);
    else if (C.cy) galerkin_node<FINE, 0, 1>(f0, F, C, I, J, out);
    else galerkin_node<FINE, 0, 0>(f0, F, C, I, J, out);
}

// Builds every coarse level's Galerkin stencil and clears its x planes
// (their padding ring stays zero: only interior nodes are written later).
__device__ void mg_setup(const Fine& f0, float* base, const MgShape& S)
{
    for (int l = 1; l <= S.levels; ++l) {
        const MgLevel C = mg_level(base, S, l);
        const MgLevel F = l > 1 ? mg_level(base, S, l - 1) : C;
        for (int t = threadIdx.x; t < C.plane; t += blockDim.x) C.x[t] = make_float2(0.f, 0.f);
        for (int t = threadIdx.x; t < C.nx * C.ny; t += blockDim.x) {
            const int I = 1 + t % C.nx, J = 1 + t / C.nx;
            float st[9];
            if (l == 1) galerkin_node_any<true>(f0, F, C, I, J, st);
            else galerkin_node_any<false>(f0, F, C, I, J, st);
            const int q = C.idx(I, J);
#pragma unroll
            for (int k = 0; k < 9; ++k) C.a[k * C.plane + q] = st[k];
        }
        __syncthreads();
    }
}

// One Gauss-Seidel colour of a nine-point level: nodes with I % 2 == ci and
// J % 2 == cj take x = (b - sum of the off-centre terms) / a_centre.
__device__ __forceinline__ void gs9_colour(const MgLevel& L, int ci, int cj)
{
    const int hx = (L.nx - ci + 1) / 2 + 1, hy = (L.ny - cj + 1) / 2 + 1;  // covers 1..nx
    for (int t = threadIdx.x; t < hx * hy; t += blockDim.x) {
        const int I = ci + 2 * (t % hx), J = cj + 2 * (t / hx);
        if (I < 1 || I > L.nx || J < 1 || J > L.ny) continue;
        const int q = L.idx(I, J);
        float2 acc = L.b[q];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            if (k == 4) continue;
            const float c = L.a[k * L.plane + q];
            const float2 v = L.x[q + ((k / 3) - 1) * L.pitch + (k % 3) - 1];
            acc.x -= c * v.x;
            acc.y -= c * v.y;
        }
        const float d = 1.f / L.a[4 * L.plane + q];
        L.x[q] = make_float2(acc.x * d, acc.y * d);
    }
    __syncthreads();
}

// t = b - A x on a nine-point level, then b of the next level = P^T t and
// its x = 0.
__device__ void mg_restrict9(const MgLevel& L, const MgLevel& C)
{
    for (int t = threadIdx.x; t < L.nx * L.ny; t += blockDim.x) {
        const int I = 1 + t % L.nx, J = 1 + t / L.nx;
        const int q = L.idx(I, J);
        float2 acc = L.b[q];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float c = L.a[k * L.plane + q];
            const float2 v = L.x[q + ((k / 3) - 1) * L.pitch + (k % 3) - 1];
            acc.x -= c * v.x;
            acc.y -= c * v.y;
        }
        L.t[q] = acc;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < C.nx * C.ny; t += blockDim.x) {
        const int I = 1 + t % C.nx, J = 1 + t / C.nx;
        const int ci = C.cx ? 2 * I : I, cj = C.cy ? 2 * J : J;
        float2 acc = make_float2(0.f, 0.f);
        for (int b = -1; b <= 1; ++b) {
            const float wb = pw(b, C.cy);
            const int fj = cj + b;
            if (wb == 0.f || fj < 1 || fj > L.ny) continue;
            for (int a = -1; a <= 1; ++a) {
                const float wa = pw(a, C.cx);
                const int fi = ci + a;
                if (wa == 0.f || fi < 1 || fi > L.nx) continue;
                const float2 v = L.t[L.idx(fi, fj)];
                acc.x += wa * wb * v.x;
                acc.y += wa * wb * v.y;
            }
        }
        const int q = C.idx(I, J);
        C.b[q] = acc;
        C.x[q] = make_float2(0.f, 0.f);
    }
    __syncthreads();
}

// x_F += P x_C on a nine-point level F (the coarse x planes have a zero ring).
__device__ void mg_prolong9(const MgLevel& F, const MgLevel& C)
{
    for (int t = threadIdx.x; t < F.nx * F.ny; t += blockDim.x) {
        const int I = 1 + t % F.nx, J = 1 + t / F.nx;
        const float2 c = mg_interp(C, I, J);
        float2& x = F.x[F.idx(I, J)];
        x.x += c.x;
        x.y += c.y;
    }
    __syncthreads();
}

// The coarsest level (at most MG_COARSEST nodes): `sweeps` damped Jacobi
// sweeps from x = 0 by warp 0, one node per lane.  The iterate stays in
// registers and each sweep reads the neighbours' values by warp shuffles (a
// neighbour on the ring reads 0); only the result goes to memory.
__device__ void mg_coarsest(const MgLevel& L, int sweeps)
{
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const bool mine = lane < L.nx * L.ny;
        const int I = mine ? 1 + lane % L.nx : 1, J = mine ? 1 + lane / L.nx : 1;
        const int q = L.idx(I, J);
        float a[9];
        int src[9];
        bool in[9];
        float2 b = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int In = I + k % 3 - 1, Jn = J + k / 3 - 1;
            in[k] = mine && In >= 1 && In <= L.nx && Jn >= 1 && Jn <= L.ny;
            src[k] = in[k] ? (In - 1) + (Jn - 1) * L.nx : lane;
        }
        if (mine) {
#pragma unroll
            for (int k = 0; k < 9; ++k) a[k] = L.a[k * L.plane + q];
            b = L.b[q];
        } else {
#pragma unroll
            for (int k = 0; k < 9; ++k) a[k] = 0.f;
            a[4] = 1.f;
        }
        const float w = 0.8f / a[4];
        float2 x = make_float2(0.f, 0.f);
        for (int s = 0; s < sweeps; ++s) {
            float2 r = b;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                float2 v;
                v.x = __shfl_sync(0xffffffffu, x.x, src[k]);
                v.y = __shfl_sync(0xffffffffu, x.y, src[k]);
                if (!in[k]) v = make_float2(0.f, 0.f);
                r.x -= a[k] * v.x;
                r.y -= a[k] * v.y;
            }
            if (mine) x = make_float2(x.x + w * r.x, x.y + w * r.y);
        }
        if (mine) L.x[q] = x;
    }
    __syncthreads();
}

// One red-black Gauss-Seidel colour on level 0 ((I + J) % 2 == colour) for
// A z = r: z = (r + sum_nbr c z_nbr) / (sum c).  z is zero on the ring.
__device__ __forceinline__ void fine_rb(const Fine& f, const Work& W, int colour)
{
    const int hx = (f.nx + 1) / 2;
    for (int t = threadIdx.x; t < hx * f.ny; t += blockDim.x) {
        const int J = 1 + t / hx;
        const int I = 1 + ((1 + J + colour) & 1) + 2 * (t % hx);
        if (I > f.nx) continue;
        float e, w, nn, so;
        f.c4(I, J, e, w, nn, so);
        const int64_t g = f.id(I, J);
        const float2 r = W.r[g];
        const float2 ze = W.z[g + 1], zw = W.z[g - 1], zn = W.z[g + f.n], zs = W.z[g - f.n];
        const float di = W.dinv[g];
        W.z[g] = make_float2((r.x + e * ze.x + w * zw.x + nn * zn.x + so * zs.x) * di,
                             (r.y + e * ze.y + w * zw.y + nn * zn.y + so * zs.y) * di);
    }
    __syncthreads();
}

// The cycle's first red sweep, from z = 0: every black neighbour is still
// zero, so the update is z = (r + 0) / (sum c), read from r and the diagonal
// alone (the + 0 turns a -0 into +0, as adding the zero products does).
__device__ __forceinline__ void fine_red_from_zero(const Fine& f, const Work& W)
{
    const int hx = (f.nx + 1) / 2;
    for (int t = threadIdx.x; t < hx * f.ny; t += blockDim.x) {
        const int J = 1 + t / hx;
        const int I = 1 + ((1 + J) & 1) + 2 * (t % hx);
        if (I > f.nx) continue;
        const int64_t g = f.id(I, J);
        const float2 r = W.r[g];
        const float di = W.dinv[g];
        W.z[g] = make_float2((r.x + 0.f) * di, (r.y + 0.f) * di);
    }
    __syncthreads();
}

// t = r - A z on level 0 (into the q workspace), then level 1: b = P^T t, x = 0.
__device__ void fine_restrict(const Fine& f, const Work& W, const MgLevel& C)
{
    for (int t = threadIdx.x; t < f.nx * f.ny; t += blockDim.x) {
        const int I = 1 + t % f.nx, J = 1 + t / f.nx;
        float e, w, nn, so;
        f.c4(I, J, e, w, nn, so);
        const int64_t g = f.id(I, J);
        const float2 r = W.r[g], z = W.z[g];
        const float2 ze = W.z[g + 1], zw = W.z[g - 1], zn = W.z[g + f.n], zs = W.z[g - f.n];
        const float d = e + w + nn + so;
        W.q[g] = make_float2(r.x - (d * z.x - (e * ze.x + w * zw.x + nn * zn.x + so * zs.x)),
                             r.y - (d * z.y - (e * ze.y + w * zw.y + nn * zn.y + so * zs.y)));
    }
    __syncthreads();
    for (int t = threadIdx.x; t < C.nx * C.ny; t += blockDim.x) {
        const int I = 1 + t % C.nx, J = 1 + t / C.nx;
        const int ci = C.cx ? 2 * I : I, cj = C.cy ? 2 * J : J;
        float2 acc = make_float2(0.f, 0.f);
        for (int b = -1; b <= 1; ++b) {
            const float wb = pw(b, C.cy);
            const int fj = cj + b;
            if (wb == 0.f || fj < 1 || fj > f.ny) continue;
            for (int a = -1; a <= 1; ++a) {
                const float wa = pw(a, C.cx);
                const int fi = ci + a;
                if (wa == 0.f || fi < 1 || fi > f.nx) continue;
                const float2 v = W.q[f.id(fi, fj)];
                acc.x += wa * wb * v.x;
                acc.y += wa * wb * v.y;
            }
        }
        const int q = C.idx(I, J);
        C.b[q] = acc;
        C.x[q] = make_float2(0.f, 0.f);
    }
    __syncthreads();
}

// z += P x_1 on level 0.
__device__ void fine_prolong(const Fine& f, const Work& W, const MgLevel& C)
{
    for (int t = threadIdx.x; t < f.nx * f.ny; t += blockDim.x) {
        const int I = 1 + t % f.nx, J = 1 + t / f.nx;
        const float2 c = mg_interp(C, I, J);
        float2& z = W.z[f.id(I, J)];
        z.x += c.x;
        z.y += c.y;
    }
    __syncthreads();
}

// z = M^-1 r: one V-cycle from z = 0.
__device__ void mg_vcycle(const Fine& f, const Work& W, float* base, const MgShape& S)
{
    // pre-smoothing on level 0 from z = 0: red (its black neighbours are
    // zero, so it reads none), then black, which writes every black node
    fine_red_from_zero(f, W);
    fine_rb(f, W, 1);
    if (S.levels > 0) {
        fine_restrict(f, W, mg_level(base, S, 1));
        for (int l = 1; l < S.levels; ++l) {
            const MgLevel L = mg_level(base, S, l);
            gs9_colour(L, 0, 0);
            gs9_colour(L, 1, 0);
            gs9_colour(L, 0, 1);
            gs9_colour(L, 1, 1);
            mg_restrict9(L, mg_level(base, S, l + 1));
        }
        const MgLevel Lc = mg_level(base, S, S.levels);
        mg_coarsest(Lc, min(96, 4 * (Lc.nx + Lc.ny) + 8));
        for (int l = S.levels - 1; l >= 1; --l) {
            const MgLevel L = mg_level(base, S, l);
            mg_prolong9(L, mg_level(base, S, l + 1));
            gs9_colour(L, 1, 1);
            gs9_colour(L, 0, 1);
            gs9_colour(L, 1, 0);
            gs9_colour(L, 0, 0);
        }
        fine_prolong(f, W, mg_level(base, S, 1));
    }
    // post-smoothing in the reverse colour order: black, then red
    fine_rb(f, W, 1);
    fine_rb(f, W, 0);
}

}  // namespace
}  // namespace sdd
