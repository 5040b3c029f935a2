// Interface Monte Carlo of the SDD mesh generator (Bihlo & Haynes, §2.1-2.2):
// Euler-Maruyama paths of dX = grad(ln c) dt + sqrt(2) dW from each interface
// node, exit test at the end of each step, score = boundary map at the exit
// point (linear interpolation of the per-edge tables), per-node sums.
//
// Work decomposition.  A work item is one chunk of `chunk` consecutive paths
// of one node of one mesh.  A persistent grid of warps pulls items from an
// atomic counter; inside an item the 32 lanes each run one path and, when
// paths exit, the freed lanes take the next paths of the item in lane order
// (ballot + popc), so lanes stay busy until the item runs dry.  The
// assignment of paths to lanes depends only on the item, so every item's
// sums, and the per-node sums built from them in chunk order, are bitwise
// reproducible whatever the launch order or the other meshes in a batch.
//
// Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed,
// counter = (step/2, path, node, 0); one call gives the four normals of two
// consecutive steps by the Box-Muller transform.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "sdd_internal.h"

namespace sdd {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int MC_THREADS = 256;          // threads per block of the path kernels (at most)
// Minimum resident blocks per SM requested from the register allocator: the
// per-family FP32-stepping kernels fit 80 registers without spills at 3
// blocks of 256, measured fastest against 4 and 2 blocks (64, 128 registers).
// The single-mesh constant-step kernels of the ring, ridge and table
// densities run blocks of 128 instead: 8 per SM (64 registers, no spills,
// 32 warps) without the bridge test, measured +1.2%, +4.7% and +11.3% over 3
// blocks of 256; 7 per SM (72 registers) with the test, which spills at 64.
// The exponential-step kernel lost 1.3% with narrow blocks and the batch
// kernels gained nothing.
#ifndef SDD_MC_MIN_BLOCKS_F32
#define SDD_MC_MIN_BLOCKS_F32 3
#endif
#ifndef SDD_MC_MIN_BLOCKS_F64
#define SDD_MC_MIN_BLOCKS_F64 1
#endif
// FP32 stepping, single-mesh kernels of the lighter densities: draw each step
// pair's Philox block one pair ahead (measured +0.5% on the ring kernel; the
// batch kernels lost 3% with it).
#ifndef SDD_PIPELINE_RNG
#define SDD_PIPELINE_RNG 1
#endif

// ------------------------------------------------------------- Philox ----
// Philox4x32-10: ten rounds of two 32x32->64 multiplies (multipliers M0, M1)
// and a Feistel-like xor/permute, the key bumped by (W0, W1) between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint32_t k0, uint32_t k1)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)M0 * x.x;   // 32x32 -> 64
        const unsigned long long p1 = (unsigned long long)M1 * x.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        x = make_uint4(hi1 ^ x.y ^ k0, lo1, hi0 ^ x.w ^ k1, lo0);
        k0 += W0;
        k1 += W1;
    }
    return x;
}

// ------------------------------------------ fast FP32 hardware approximations
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sin_approx(float x)
{
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float cos_approx(float x)
{
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr float TWO_PI_F = 6.28318530717958647692f;
constexpr double PI_D = 3.14159265358979323846;

// Box-Muller, FP32.  Uniforms U = (floor(r / 2^9) + 1/2) 2^-23 are exact in
// FP32 and lie in (0,1); the angle 2 pi U is taken as 2 pi (U - 1/2) + pi,
// i.e. (cos, sin)(2 pi U) = -(cos, sin)(2 pi (U - 1/2)), which keeps the
// argument of the hardware sine/cosine in [-pi, pi] (the sign goes into nr);
// the angle's uniform drops the half step (see box_muller_f32_step).
__device__ __forceinline__ float uniform23(uint32_t r)
{
    // 1 + floor(r/2^9) 2^-23 in [1,2), minus (1 - 2^-24): exact.
    return __uint_as_float((r >> 9) + 0x3f800000u) - 0.99999994039535522461f;
}

// Box-Muller, FP32, returning the noise increment of a step in factored form:
// sqrt(2 dt) (z0, z1) = (nr cos, nr sin), nr = -sqrt(-4 dt ln ua) and
// (cos, sin) of 2 pi (ub - 1/2); c4dt = -4 dt ln 2.  The caller adds each
// component with one fused multiply-add.
__device__ __forceinline__ void box_muller_f32_step(uint32_t ra, uint32_t rb, float c4dt,
                                                    float& nr, float& cz, float& sz)
{
    const float ua = uniform23(ra);
    const float v = c4dt * lg2_approx(ua);                  // -4 dt ln ua > 0
    nr = -sqrt_approx(v);
    // angle 2 pi (floor(rb / 2^9) 2^-23 - 1/2), exact before the multiply: the
    // grid of the FP64 angle shifted by half an FP32 step, a fixed rotation by
    // 2 pi 2^-24 that leaves the distribution of the normal pair unchanged
    const float ang = TWO_PI_F * (__uint_as_float((rb >> 9) + 0x3f800000u) - 1.5f);
    cz = cos_approx(ang);
    sz = sin_approx(ang);
}

// Exponential time stepping (§2.2): the lengths of steps 4q .. 4q+3 are dt E
// with E = -ln U, U from words 0..3 of Philox counter (q, path, node, 2).
// FP64: U = (r + 1/2) 2^-32.  FP32: returns
// E / ln 2 = -log2 U with the FP32 uniform, clamped at 0 (the approximate
// log2 of a U next to 1 may land on the wrong side of 0).
__device__ __forceinline__ double exp_unit_f64(uint32_t r)
{
    return -log(((double)r + 0.5) * 0x1p-32);
}
__device__ __forceinline__ float exp_unit_log2_f32(uint32_t r)
{
    return fmaxf(-lg2_approx(uniform23(r)), 0.0f);
}

// Box-Muller, FP64 with CUDA's double-precision log / sqrt / sincospi.
__device__ __forceinline__ void box_muller_f64(uint32_t ra, uint32_t rb, double& z0, double& z1)
{
    const double ua = ((double)ra + 0.5) * 0x1p-32;
    const double ub = ((double)rb + 0.5) * 0x1p-32;
    const double R = sqrt(-2.0 * log(ua));
    double s, c;
    sincospi(2.0 * ub, &s, &c);
    z0 = R * c;
    z1 = R * s;
}

// ----------------------------------------------------- densities, FP32 ----
// Each FP32 density gives the drift half of an Euler-Maruyama step:
// advance(s, t, f) = (s, t) + b f dt with b = grad ln c = sgn grad(w)/w
// (c = w^sgn), f dt folded into the last multiplication; f = 1 for constant
// steps (the multiplication by the constant 1 folds away), f = h/dt for a
// step of length h (exponential time stepping).
// BUMPS: pf[8b..8b+6] = A, cs, ct, ks log2 e, kt log2 e, -2 ks, -2 kt.
template <int NB>
struct BumpsF32 {
    static constexpr bool kLight = NB <= 2;   // registers to spare for a Philox block
    float p[NB][7];
    float sdt;                  // sgn * dt
    __device__ void load(const MeshDev& M)
    {
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int q = 0; q < 7; ++q) p[b][q] = M.pf[8 * b + q];
        sdt = (float)(M.sgn * M.dt);
    }
    __device__ __forceinline__ void advance(float s, float t, float& as, float& at,
                                            float fdt = 1.0f) const
    {
        float w = 1.0f, gs = 0.0f, gt = 0.0f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const float ds = s - p[b][1], dtt = t - p[b][2];
            const float ex = -fmaf(p[b][3] * ds, ds, p[b][4] * dtt * dtt);
            const float e = p[b][0] * ex2_approx(ex);
            w += e;
            gs = fmaf(e * p[b][5], ds, gs);
            gt = fmaf(e * p[b][6], dtt, gt);
        }
        const float inv = (sdt * fdt) * rcp_approx(w);
        as = fmaf(gs, inv, s);
        at = fmaf(gt, inv, t);
    }
};

// RING: pf = cs, ct, r0, -2 k log2 e, 4 A, sgn * (-8 A k).
// With e = exp(-2|u|), u = k (r - r0):  (dw/dr) / w = -8 A k sign(u) e (1 - e)
// / ((1 + e)((1 + e)^2 + 4 A e)), and b = sgn (dw/dr)/w (s - cs, t - ct)/r.
struct RingF32 {
    static constexpr bool kLight = true;
    float cs, ct, r0, c1, A4, Kdt;
    __device__ void load(const MeshDev& M)
    {
        cs = M.pf[0]; ct = M.pf[1]; r0 = M.pf[2]; c1 = M.pf[3]; A4 = M.pf[4];
        Kdt = (float)((double)M.pf[5] * M.dt);
    }
    __device__ __forceinline__ void advance(float s, float t, float& as, float& at,
                                            float fdt = 1.0f) const
    {
        const float ds = s - cs, dtt = t - ct;
        const float r2 = fmaf(ds, ds, fmaf(dtt, dtt, 1e-30f));   // > 0 at the centre too
        const float rinv = rsqrt_approx(r2);
        const float u = fmaf(r2, rinv, -r0);
        const float e = ex2_approx(c1 * fabsf(u));
        const float ope = 1.0f + e;
        const float D = ope * fmaf(ope, ope, A4 * e);
        const float num = copysignf(fmaf(-e, e, e), u) * rinv;
        const float f = ((Kdt * fdt) * num) * rcp_approx(D);
        as = fmaf(f, ds, s);
        at = fmaf(f, dtt, t);
    }
};

// RIDGE: pf = A, k log2 e, t0, a, f, -2 k, -2 pi a f.
// v = t - t0 - a sin(2 pi f s); w = 1 + A exp(-k v^2);
// dw/dt = e (-2 k v), dw/ds = dw/dt (-2 pi a f cos(2 pi f s)).
struct RidgeF32 {
    static constexpr bool kLight = true;
    float A, kl, t0, a, f, m2k, m2paf, sdt;
    __device__ void load(const MeshDev& M)
    {
        A = M.pf[0]; kl = M.pf[1]; t0 = M.pf[2]; a = M.pf[3]; f = M.pf[4];
        m2k = M.pf[5]; m2paf = M.pf[6]; sdt = (float)(M.sgn * M.dt);
    }
    __device__ __forceinline__ void advance(float s, float t, float& as, float& at,
                                            float fdt = 1.0f) const
    {
        const float fr = f * s;
        const float x = TWO_PI_F * (fr - rintf(fr));           // in [-pi, pi]
        const float sn = sin_approx(x), cn = cos_approx(x);
        const float v = t - t0 - a * sn;
        const float e = A * ex2_approx(-kl * v * v);
        const float inv = (sdt * fdt) * rcp_approx(1.0f + e);
        const float gt = e * m2k * v;
        at = fmaf(gt, inv, t);
        as = fmaf(gt * (m2paf * cn), inv, s);
    }
};

// TABLE: w = exp(L), L the bilinear interpolant of a table of ln w at the
// tn x tn nodes; the drift is sgn grad L, the interpolant's exact cellwise
// gradient: with (fa, fb) the position in its cell, dL/ds = c1 + c3 fb and
// dL/dt = c2 + c3 fa, (c1, c2, c3) one 16-byte record per cell read through
// the read-only cache (one gather per drift evaluation).  The position is
// clamped into [0, tn-1) cells; the cell index is formed in FP32 (exact for
// tn <= 4097).
struct TableF32 {
    static constexpr bool kLight = true;
    const float4* cell;
    float m, xmax, sdt;
    __device__ void load(const MeshDev& M)
    {
        cell = M.cell32;
        m = (float)(M.tn - 1);
        xmax = __int_as_float(__float_as_int(m) - 1);      // largest float below tn - 1
        sdt = (float)(M.sgn * M.dt);
    }
    __device__ __forceinline__ void advance(float s, float t, float& as, float& at,
                                            float fdt = 1.0f) const
    {
        const float x = fminf(fmaxf(s * m, 0.0f), xmax), y = fminf(fmaxf(t * m, 0.0f), xmax);
        const float xf = floorf(x), yf = floorf(y);
        const float fa = x - xf, fb = y - yf;
        const float4 c = __ldg(cell + __float2int_rz(fmaf(yf, m, xf)));
        const float k = sdt * fdt;
        as = fmaf(k, fmaf(c.z, fb, c.x), s);
        at = fmaf(k, fmaf(c.z, fa, c.y), t);
    }
};

// ----------------------------------------------------- densities, FP64 ----
struct BumpsF64 {
    const double* p;
    int nb;
    double sgn;
    __device__ void load(const MeshDev& M) { p = M.pd; nb = M.nb; sgn = M.sgn; }
    __device__ __forceinline__ void drift(double s, double t, double& bs, double& bt) const
    {
        double w = 1.0, gs = 0.0, gt = 0.0;
        for (int b = 0; b < nb; ++b) {
            const double* q = p + 1 + 5 * b;
            const double A = q[0], cs = q[1], ct = q[2], ks = q[3], kt = q[4];
            const double ds = s - cs, dtt = t - ct;
            const double e = A * exp(-(ks * ds * ds + kt * dtt * dtt));
            w += e;
            gs += e * (-2.0 * ks * ds);
            gt += e * (-2.0 * kt * dtt);
        }
        bs = sgn * gs / w;
        bt = sgn * gt / w;
    }
};

struct RingF64 {
    double A, cs, ct, k, r0, sgn;
    __device__ void load(const MeshDev& M)
    {
        A = M.pd[0]; cs = M.pd[1]; ct = M.pd[2]; k = M.pd[3]; r0 = M.pd[4]; sgn = M.sgn;
    }
    __device__ __forceinline__ void drift(double s, double t, double& bs, double& bt) const
    {
        const double ds = s - cs, dtt = t - ct;
        const double r = sqrt(ds * ds + dtt * dtt);
        if (r == 0.0) { bs = 0.0; bt = 0.0; return; }
        const double u = k * (r - r0);
        const double e = exp(-2.0 * fabs(u));
        const double ope = 1.0 + e;
        const double D = ope * (ope * ope + 4.0 * A * e);
        const double g = sgn * (-8.0 * A * k) * copysign(e * (1.0 - e), u) / (D * r);
        bs = g * ds;
        bt = g * dtt;
    }
};

struct RidgeF64 {
    double A, k, t0, a, f, sgn;
    __device__ void load(const MeshDev& M)
    {
        A = M.pd[0]; k = M.pd[1]; t0 = M.pd[2]; a = M.pd[3]; f = M.pd[4]; sgn = M.sgn;
    }
    __device__ __forceinline__ void drift(double s, double t, double& bs, double& bt) const
    {
        double sn, cn;
        sincospi(2.0 * f * s, &sn, &cn);
        const double v = t - t0 - a * sn;
        const double e = A * exp(-k * v * v);
        const double w = 1.0 + e;
        const double gt = e * (-2.0 * k * v);
        const double gs = gt * (-2.0 * PI_D * a * f * cn);
        bs = sgn * gs / w;
        bt = sgn * gt / w;
    }
};

// ------------------------------------------------------ exit and score ----
// Edge crossed by the step x -> y (some coordinate of y outside (0,1)) and the
// tangential coordinate of the exit point: for each violated side
// theta = (x_d - side) / (x_d - y_d); the smallest theta wins, an exact tie
// going to the s-sides; the tangential coordinate is clamped to [0,1].
// Edges: 0 bottom (t=0), 1 top (t=1), 2 left (s=0), 3 right (s=1).
template <typename R>
__device__ __forceinline__ int exit_edge(R xs, R xt, R ys, R yt, R& tau)
{
    int es = -1, et = -1;
    R ths = R(2), tht = R(2);
    if (ys <= R(0)) { es = 2; ths = xs / (xs - ys); }
    else if (ys >= R(1)) { es = 3; ths = (xs - R(1)) / (xs - ys); }
    if (yt <= R(0)) { et = 0; tht = xt / (xt - yt); }
    else if (yt >= R(1)) { et = 1; tht = (xt - R(1)) / (xt - yt); }
    if (es >= 0 && (et < 0 || ths <= tht)) {
        tau = fmin(fmax(xt + ths * (yt - xt), R(0)), R(1));
        return es;
    }
    tau = fmin(fmax(xs + tht * (ys - xs), R(0)), R(1));
    return et;
}

// Nearest side of an interior point (first minimum in the order s=0, s=1,
// t=0, t=1) and the tangential coordinate of its projection; used for paths
// stopped by the step cap.
template <typename R>
__device__ __forceinline__ int nearest_edge(R s, R t, R& tau)
{
    R d = s;
    int e = 2;
    tau = t;
    if (R(1) - s < d) { d = R(1) - s; e = 3; }
    if (t < d) { d = t; e = 0; tau = s; }
    if (R(1) - t < d) { e = 1; tau = s; }
    return e;
}

// Brownian-bridge exit test of a step x -> y that ended inside (§2.2, after
// Gobet): side m is crossed with probability p_m = exp(-d_m(x) d_m(y) / dt)
// (noise sqrt(2) dW), decided by U_m of Philox counter (k, path, node, 1) in
// the side order s=0, s=1, t=0, t=1 (edges 2, 3, 0, 1).  No side can be
// crossed when every product is >= qmax, and then no uniforms are drawn:
// with FP64 uniforms (smallest 2^-33) qmax = 23 dt gives p < 1.03e-10 <
// 2^-33; with the FP32 uniforms of uniform23 (smallest 2^-24) qmax = 16.7 dt
// gives p <= 2^-24.09 < 2^-24.  Either way U < p is impossible there, so the
// cut changes no decision.  Returns the edge and the tangential coordinate of the
// exit point (mean of the step's two), or -1.
template <typename R, class Keys>
__device__ __forceinline__ int bridge_exit_inl(R xs, R xt, R ys, R yt, R inv_dt, R qmax,
                                               const Keys& philox, uint32_t k, uint32_t path,
                                               uint32_t node, R& tau, bool& tie)
{
    const R q[4] = {xs * ys, (R(1) - xs) * (R(1) - ys), xt * yt, (R(1) - xt) * (R(1) - yt)};
    if (!((q[0] < qmax) | (q[1] < qmax) | (q[2] < qmax) | (q[3] < qmax))) return -1;
    const uint4 r4 = philox(make_uint4(k, path, node, 1u));
    const uint32_t rr[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        if (!(q[m] < qmax)) continue;
        R p, u;
        if constexpr (sizeof(R) == 8) {
            p = exp(-q[m] * inv_dt);
            u = ((double)rr[m] + 0.5) * 0x1p-32;
            if (fabs(u - p) < 1e-12) tie = true;
        } else {
            p = ex2_approx(-q[m] * inv_dt * 1.44269504088896340736f);
            u = uniform23(rr[m]);
        }
        if (u < p) {
            tau = m < 2 ? fmin(fmax(R(0.5) * (xt + yt), R(0)), R(1))
                        : fmin(fmax(R(0.5) * (xs + ys), R(0)), R(1));
            return m == 0 ? 2 : m == 1 ? 3 : m == 2 ? 0 : 1;
        }
    }
    return -1;
}

// The same test as a called function: the FP64 runner and the FP32 kernels
// without the test keep it out of their register allocation.
template <typename R, class Keys>
__device__ __noinline__ int bridge_exit(R xs, R xt, R ys, R yt, R inv_dt, R qmax, const Keys& philox,
                                        uint32_t k, uint32_t path, uint32_t node, R& tau, bool& tie)
{
    return bridge_exit_inl<R>(xs, xt, ys, yt, inv_dt, qmax, philox, k, path, node, tau, tie);
}

// Linear interpolation in a table of n values at tau_j = j/(n-1), in FP64.
__device__ __forceinline__ double lookup(const double* __restrict__ T, int n, double tau)
{
    const double x = tau * (double)(n - 1);
    int j = (int)floor(x);
    j = min(max(j, 0), n - 2);
    const double fr = x - (double)j;
    const double a = __ldg(T + j), b = __ldg(T + j + 1);
    return a + fr * (b - a);
}

// --------------------------------------------------- compensated sums ----
__device__ __forceinline__ void two_sum_add(double& hi, double& lo, double x)
{
    const double s = hi + x;
    const double bb = s - hi;
    lo += (hi - (s - bb)) + (x - bb);
    hi = s;
}

// Per-lane accumulators live in shared memory (they are touched once per
// path, not per step), one column per thread, so the step loop keeps only the
// path state in registers.
struct AccSmem {
    double v[12][MC_THREADS];   // s_hi[2] s_lo[2] q_hi[2] q_lo[2] st[2] qt[2]
};

__device__ __forceinline__ void acc_zero(AccSmem& A, int tid)
{
#pragma unroll
    for (int q = 0; q < 12; ++q) A.v[q][tid] = 0.0;
}

// Adds d = F - X0 of one path: compensated sums over non-tie paths, plain sums
// over tie-flagged paths.
__device__ __forceinline__ void acc_add(AccSmem& A, int tid, double d0, double d1, bool tie)
{
    if (!tie) {
        double h, l;
        h = A.v[0][tid]; l = A.v[2][tid]; two_sum_add(h, l, d0); A.v[0][tid] = h; A.v[2][tid] = l;
        h = A.v[1][tid]; l = A.v[3][tid]; two_sum_add(h, l, d1); A.v[1][tid] = h; A.v[3][tid] = l;
        h = A.v[4][tid]; l = A.v[6][tid]; two_sum_add(h, l, d0 * d0); A.v[4][tid] = h; A.v[6][tid] = l;
        h = A.v[5][tid]; l = A.v[7][tid]; two_sum_add(h, l, d1 * d1); A.v[5][tid] = h; A.v[7][tid] = l;
    } else {
        A.v[8][tid] += d0;
        A.v[9][tid] += d1;
        A.v[10][tid] += d0 * d0;
        A.v[11][tid] += d1 * d1;
    }
}

// Butterfly over the warp of the lane sums; lane 0 writes the item's slot.
__device__ void acc_write_slot(const AccSmem& A, int tid, int lane, uint32_t ties, uint32_t caps,
                               unsigned long long steps, uint32_t paths, Slot* __restrict__ out)
{
    double v[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) v[q] = A.v[q][tid];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            // (hi, lo) pairs: (v[q], v[q + 2]) for q = 0, 1 and (v[q + 2], v[q + 4]) for q = 2, 3
            const int hq = q < 2 ? q : q + 2, lq = hq + 2;
            const double oh = __shfl_xor_sync(FULL, v[hq], off);
            const double ol = __shfl_xor_sync(FULL, v[lq], off);
            v[lq] += ol;
            two_sum_add(v[hq], v[lq], oh);
        }
#pragma unroll
        for (int q = 8; q < 12; ++q) v[q] += __shfl_xor_sync(FULL, v[q], off);
        ties += __shfl_xor_sync(FULL, ties, off);
        caps += __shfl_xor_sync(FULL, caps, off);
        steps += __shfl_xor_sync(FULL, steps, off);
        paths += __shfl_xor_sync(FULL, paths, off);
    }
    if (lane == 0) {
        Slot sl;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            sl.s_hi[c] = v[c]; sl.s_lo[c] = v[2 + c];
            sl.q_hi[c] = v[4 + c]; sl.q_lo[c] = v[6 + c];
            sl.st[c] = v[8 + c]; sl.qt[c] = v[10 + c];
        }
        sl.ties = ties;
        sl.caps = caps;
        sl.steps = steps;
        sl.paths = paths;
#pragma unroll
        for (int c = 0; c < 2; ++c) sl.fx_s[c] = sl.fx_q[c] = 0;
        *out = sl;
    }
}

// TABLE, FP64: the same interpolant, the drift sgn grad L in the oracle's
// order of operations.
struct TableF64 {
    const double* tab;
    int tn;
    double m, sgn;
    __device__ void load(const MeshDev& M)
    {
        tab = M.tab64;
        tn = M.tn;
        m = (double)(M.tn - 1);
        sgn = M.sgn;
    }
    __device__ __forceinline__ void drift(double s, double t, double& bs, double& bt) const
    {
        const double x = s * m, y = t * m;
        const int a = min(max((int)floor(x), 0), tn - 2), b = min(max((int)floor(y), 0), tn - 2);
        const double fa = x - (double)a, fb = y - (double)b;
        const double* r0 = tab + b * tn + a;
        const double L00 = __ldg(r0), L10 = __ldg(r0 + 1);
        const double L01 = __ldg(r0 + tn), L11 = __ldg(r0 + tn + 1);
        const double Ls = ((1.0 - fb) * (L10 - L00) + fb * (L11 - L01)) * m;
        const double Lt = ((1.0 - fa) * (L01 - L00) + fa * (L11 - L10)) * m;
        bs = sgn * Ls;
        bt = sgn * Lt;
    }
};

template <int PREC> struct RealOf { using T = double; };
template <> struct RealOf<SDD_FP32_STEP> { using T = float; };

// Philox keys.  Batched FP64 launches carry one key per mesh and advance it
// by the Weyl constants round by round; single-mesh launches take the ten
// round keys precomputed on the host from the kernel parameters, so they
// enter the xors as constant operands.
struct RegKeys {
    uint32_t k0, k1;
    __device__ __forceinline__ uint4 operator()(uint4 x) const { return philox4x32_10(x, k0, k1); }
};
// Batched FP32 launches: the ten round keys of the warp's current mesh in
// the warp's slot of shared memory (written when the warp turns to a mesh),
// read as operands instead of being advanced in registers (the batch rate
// rose 7%, to the single-mesh kernels' rate).
struct SmemKeys {
    const uint32_t* rk;
    __device__ __forceinline__ uint4 operator()(uint4 x) const
    {
        const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            const unsigned long long p0 = (unsigned long long)M0 * x.x;
            const unsigned long long p1 = (unsigned long long)M1 * x.z;
            const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
            const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
            x = make_uint4(hi1 ^ x.y ^ rk[2 * r], lo1, hi0 ^ x.w ^ rk[2 * r + 1], lo0);
        }
        return x;
    }
};

struct ParamKeys {
    const uint32_t (&rk)[20];
    __device__ __forceinline__ uint4 operator()(uint4 x) const
    {
        const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            const unsigned long long p0 = (unsigned long long)M0 * x.x;
            const unsigned long long p1 = (unsigned long long)M1 * x.z;
            const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
            const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
            x = make_uint4(hi1 ^ x.y ^ rk[2 * r], lo1, hi0 ^ x.w ^ rk[2 * r + 1], lo0);
        }
        return x;
    }
};

// ------------------------------------------------------- one work item ----
// Runs the paths of chunk `chunk` of node `node`; lanes refill from the chunk
// in lane order as their paths end.  Two Euler-Maruyama steps per Philox call;
// the step cap is tested once per pair except in the pair that reaches it.
template <int PREC, class Dens, class Keys>
__device__ __forceinline__ void run_item(const MeshDev& M, const Dens& dens, const Keys& philox,
                                         uint32_t node, uint32_t chunk, Slot* __restrict__ out,
                                         AccSmem& A, int tid, int lane)
{
    using R = typename RealOf<PREC>::T;
    const int n = M.n;
    const int2 ij = M.nodes[node];
    const uint32_t nid = M.node_ids ? M.node_ids[node] : node;     // Philox counter word
    const double s0d = (double)ij.x / (double)(n - 1);
    const double t0d = (double)ij.y / (double)(n - 1);
    const R s0 = (R)s0d, t0 = (R)t0d;
    const R dtR = (R)M.dt, sq = (R)M.sqrt2dt;
    const R delta = (R)M.tie_delta;
    const uint32_t kmax = M.max_steps;
    const uint32_t p_begin = chunk * M.chunk;
    const uint32_t p_end = min(M.paths, p_begin + M.chunk);

    uint32_t path = p_begin + (uint32_t)lane;
    bool active = path < p_end;
    uint32_t cursor = p_begin + 32u;
    R xs = s0, xt = t0;      // position before the current step
    R ys = s0, yt = t0;      // position after it
    uint32_t k = 0;
    bool tie = false;
    uint32_t ties = 0, caps = 0, npaths = 0;
    unsigned long long steps = 0;
    acc_zero(A, tid);
    __syncwarp();

    const bool bridge = M.bridge != 0;
    const bool expo = M.stepper == SDD_STEP_EXPONENTIAL;
    uint4 Lq = make_uint4(0u, 0u, 0u, 0u);     // Philox block of the current four step lengths
    const R inv_dt = R(1) / dtR, qmax = R(23) * dtR;
    int bedge = -1;
    R btau = R(0);

    // One Euler-Maruyama step of length h from (xs, xt) with normals (za, zb)
    // into (ys, yt).  Returns 0 to continue, 1 on exit through the end point,
    // 2 at the step cap, 3 on a Brownian-bridge crossing (edge bedge, btau).
    auto step = [&](R za, R zb, R h, bool check_cap) -> int {
        R bs, bt;
        dens.drift(xs, xt, bs, bt);
        const R sqh = expo ? sqrt(R(2) * h) : sq;
        ys = xs + bs * h + sqh * za;
        yt = xt + bt * h + sqh * zb;
        ++k;
        if constexpr (PREC == SDD_FP64) {
            const R m = fmin(fmin(fabs(ys), fabs(R(1) - ys)), fmin(fabs(yt), fabs(R(1) - yt)));
            tie = tie || (m < delta);
        }
        if ((ys <= R(0)) | (ys >= R(1)) | (yt <= R(0)) | (yt >= R(1))) return 1;
        if (bridge) {
            bedge = bridge_exit<R>(xs, xt, ys, yt, expo ? R(1) / h : inv_dt,
                                   expo ? R(23) * h : qmax, philox, k - 1u, path, nid, btau, tie);
            if (bedge >= 0) return 3;
        }
        if (check_cap && k >= kmax) return 2;
        xs = ys;
        xt = yt;
        return 0;
    };

    for (;;) {
        int ended = 0;
        if (active) {
            const uint4 r = philox(make_uint4(k >> 1, path, nid, 0u));
            R z0, z1, z2, z3;
            if constexpr (PREC == SDD_FP64) {
                box_muller_f64(r.x, r.y, z0, z1);
                box_muller_f64(r.z, r.w, z2, z3);
            } else {
                box_muller_f32(r.x, r.y, z0, z1);
                box_muller_f32(r.z, r.w, z2, z3);
            }
            R h0 = dtR, h1 = dtR;
            if (expo) {
                // lengths of steps 4q..4q+3 from one block: words x, y for the
                // first pair of the four steps, z, w for the second
                if ((k & 2u) == 0u) Lq = philox(make_uint4(k >> 2, path, nid, 2u));
                const uint32_t wa = (k & 2u) ? Lq.z : Lq.x, wb = (k & 2u) ? Lq.w : Lq.y;
                if constexpr (PREC == SDD_FP64) {
                    h0 = dtR * exp_unit_f64(wa);
                    h1 = dtR * exp_unit_f64(wb);
                } else {
                    h0 = dtR * (exp_unit_log2_f32(wa) * 0.69314718055994530942f);
                    h1 = dtR * (exp_unit_log2_f32(wb) * 0.69314718055994530942f);
                }
            }
            if (k + 2u <= kmax) {
                ended = step(z0, z1, h0, false);
                if (!ended) ended = step(z2, z3, h1, false);
                if (!ended && k >= kmax) ended = 2;
            } else {
                ended = step(z0, z1, h0, true);
                if (!ended) ended = step(z2, z3, h1, true);
            }
            if (ended) {
                R tau = btau;                      // bridge crossing: edge and point known
                int e = ended == 1 ? exit_edge<R>(xs, xt, ys, yt, tau) : ended == 3 ? bedge : -1;
                if (e < 0) {                       // step cap (or a non-finite position)
                    e = nearest_edge<R>(ys, yt, tau);
                    ended = 2;
                }
                const double td = (double)tau;
                const double f0 = lookup(M.edges + (size_t)e * n, n, td);
                const double f1 = lookup(M.edges + (size_t)(4 + e) * n, n, td);
                acc_add(A, tid, f0 - s0d, f1 - t0d, tie);
                ties += tie ? 1u : 0u;
                caps += ended == 2 ? 1u : 0u;
                steps += k;
                ++npaths;
            }
        }
        const unsigned dm = __ballot_sync(FULL, ended != 0);
        if (dm) {
            if (ended) {
                const unsigned rank = __popc(dm & ((1u << lane) - 1u));
                path = cursor + rank;
                active = path < p_end;
                xs = s0;
                xt = t0;
                k = 0;
                tie = false;
            }
            cursor += (uint32_t)__popc(dm);
        }
        if (!__any_sync(FULL, active)) break;
    }
    __syncwarp();
    acc_write_slot(A, tid, lane, ties, caps, steps, npaths, out);
    __syncwarp();
}

template <int PREC, class Dens, class Keys>
__device__ __forceinline__ void run_with(const MeshDev& M, const Keys& keys, uint32_t node,
                                         uint32_t chunk, Slot* out, AccSmem& A, int tid, int lane)
{
    Dens d;
    d.load(M);
    run_item<PREC, Dens, Keys>(M, d, keys, node, chunk, out, A, tid, lane);
}

template <int PREC, class Keys>
__device__ __forceinline__ void dispatch(const MeshDev& M, const Keys& keys, uint32_t node,
                                         uint32_t chunk, Slot* out, AccSmem& A, int tid, int lane)
{
    static_assert(PREC == SDD_FP64, "item-at-a-time runner serves FP64 stepping");
    switch (M.family) {
        case SDD_FAMILY_RING: run_with<PREC, RingF64>(M, keys, node, chunk, out, A, tid, lane); break;
        case SDD_FAMILY_RIDGE: run_with<PREC, RidgeF64>(M, keys, node, chunk, out, A, tid, lane); break;
        case SDD_FAMILY_TABLE: run_with<PREC, TableF64>(M, keys, node, chunk, out, A, tid, lane); break;
        default: run_with<PREC, BumpsF64>(M, keys, node, chunk, out, A, tid, lane); break;
    }
}

// ----------------------------------------- FP32 stepping: path streams ----
// In FP32 stepping the lanes of a warp stream through consecutive work items
// of one mesh: when an item has handed out all its paths, the lanes that
// free up start paths of the next item while the others finish theirs, so no
// lane waits for the slowest path of an item.  Each item's sums live in one
// of four per-warp accumulator sets in shared memory until its last path has
// ended, then the set is written to the item's slot.  Scores enter the sums
// as 2^-40 fixed-point integers (|d| <= 1, so an item of at most 8192 paths
// stays below 2^53 and converts to FP64 exactly), which makes every item's
// sums exact and independent of which lane ran which path.
constexpr int N_SETS = 4;
constexpr double FX_SCALE = 1099511627776.0;        // 2^40

struct WarpAcc {
    unsigned long long s[N_SETS][2];    // sum of d, fixed point
    unsigned long long q[N_SETS][2];    // sum of d^2, fixed point
    unsigned long long steps[N_SETS];
    unsigned int caps[N_SETS];
    unsigned int paths[N_SETS];
    // warp-uniform bookkeeping of the stream (read by every lane, written by lane 0)
    unsigned long long set_item[N_SETS];
    unsigned int set_live[N_SETS];      // lanes running a path of the set's item
    unsigned int used;                  // bit s: set s holds an open item
    int cur;                            // set of the item being handed out, -1: none
    unsigned int cur_cursor, cur_end, cur_node;
    unsigned long long held;            // taken from the queue, not opened yet
    unsigned long long pending;         // first item that is not this mesh's
    int held_valid, have_pending;
};

__device__ __forceinline__ void set_zero(WarpAcc& W, int s, int lane)
{
    if (lane < 2) { W.s[s][lane] = 0ull; W.q[s][lane] = 0ull; }
    if (lane == 2) W.steps[s] = 0ull;
    if (lane == 3) { W.caps[s] = 0u; W.paths[s] = 0u; }
}

__device__ __forceinline__ void set_flush(const WarpAcc& W, int s, Slot* __restrict__ out, int lane)
{
    if (lane == 0) {
        Slot sl;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            sl.s_hi[c] = sl.s_lo[c] = sl.q_hi[c] = sl.q_lo[c] = sl.st[c] = sl.qt[c] = 0.0;
            sl.fx_s[c] = (long long)W.s[s][c];
            sl.fx_q[c] = (long long)W.q[s][c];
        }
        sl.ties = 0u;
        sl.caps = W.caps[s];
        sl.paths = W.paths[s];
        sl.steps = W.steps[s];
        sl.reserved = 0u;
        *out = sl;
    }
}

// Rare part of the stream loop, run by the whole warp when paths have ended:
// releases the ended lanes (mask dm), writes out the sets whose item is
// finished, and hands new paths to idle lanes (opening the next items from
// the queue as needed).  The new path of a lane is returned through
// the returned record (given = lanes that received a path).
struct Refill {
    unsigned given;
    uint32_t path, node;
    int set;
};

__device__ __forceinline__ Refill stream_refill_inl(const MeshDev& M, const McArgs& a, WarpAcc& W,
                                                   int lane, unsigned dm, unsigned idle,
                                                   unsigned long long mesh_end)
{
    Refill out{0u, 0u, 0u, 0};
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t C = M.chunk, cpn = M.chunks_per_node, N = M.paths;
    __syncwarp();
    unsigned live[N_SETS];
#pragma unroll
    for (int s = 0; s < N_SETS; ++s) live[s] = W.set_live[s] & ~dm;
    unsigned used = W.used;
    int cur = W.cur;
    uint32_t cursor = W.cur_cursor, end = W.cur_end, cnode = W.cur_node;
    unsigned long long held = W.held, pending = W.pending;
    bool held_valid = W.held_valid != 0, have_pending = W.have_pending != 0;
    __syncwarp();
    // close the sets whose item has no path left to hand out or running
#pragma unroll
    for (int s = 0; s < N_SETS; ++s) {
        if (((used >> s) & 1u) && live[s] == 0u && !(s == cur && cursor < end)) {
            set_flush(W, s, a.slots + W.set_item[s], lane);
            used &= ~(1u << s);
            if (s == cur) cur = -1;
        }
    }
    __syncwarp();
    unsigned given = 0u;
    unsigned want = idle;
    while (want) {
        if (cur < 0 || cursor >= end) {
            if (!held_valid) {
                if (have_pending) break;
                unsigned long long it = 0;
                if (lane == 0) it = a.item_base + atomicAdd(a.queue, 1ull);
                it = __shfl_sync(FULL, it, 0);
                if (it >= a.total_items || it >= mesh_end) {
                    pending = it;
                    have_pending = true;
                    break;
                }
                held = it;
                held_valid = true;
            }
            if ((uint32_t)((held - M.item_begin) % cpn) < M.chunk_begin) {
                held_valid = false;                    // summed by the run this one continues
                continue;
            }
            const unsigned freeb = ~used & ((1u << N_SETS) - 1u);
            if (!freeb) break;                         // all sets busy: wait for a flush
            const int s = __ffs(freeb) - 1;
            set_zero(W, s, lane);
            if (lane == 0) W.set_item[s] = held;
            __syncwarp();
            used |= 1u << s;
#pragma unroll
            for (int q = 0; q < N_SETS; ++q)
                if (q == s) live[q] = 0u;
            cur = s;
            const unsigned long long local = held - M.item_begin;
            cnode = (uint32_t)(local / cpn);
            cursor = (uint32_t)(local % cpn) * C;
            end = min(N, cursor + C);
            held_valid = false;
        }
        const uint32_t avail = end - cursor;
        const unsigned r = __popc(want & lt);
        const bool mine = ((want >> lane) & 1u) && r < avail;
        const unsigned taken = __ballot_sync(FULL, mine);
        if (mine) {
            out.path = cursor + r;
            out.node = cnode;
            out.set = cur;
        }
#pragma unroll
        for (int q = 0; q < N_SETS; ++q)
            if (q == cur) live[q] |= taken;
        cursor += (uint32_t)__popc(taken);
        want &= ~taken;
        given |= taken;
    }
    if (lane == 0) {
#pragma unroll
        for (int s = 0; s < N_SETS; ++s) W.set_live[s] = live[s];
        W.used = used;
        W.cur = cur;
        W.cur_cursor = cursor;
        W.cur_end = end;
        W.cur_node = cnode;
        W.held = held;
        W.pending = pending;
        W.held_valid = held_valid ? 1 : 0;
        W.have_pending = have_pending ? 1 : 0;
    }
    __syncwarp();
    out.given = given;
    return out;
}

// The refill as a called function (the batch kernels and the kernels with the
// bridge test, whose register allocation is tighter); the single-mesh kernels
// without the test inline it (+2% on the 257 x 257 ring workload).
__device__ __noinline__ Refill stream_refill(const MeshDev& M, const McArgs& a, WarpAcc& W,
                                             int lane, unsigned dm, unsigned idle,
                                             unsigned long long mesh_end)
{
    return stream_refill_inl(M, a, W, lane, dm, idle, mesh_end);
}

// Streams the items of mesh M starting at `first` (already taken from the
// queue).  Returns the first item taken that is not M's (the next mesh's, or
// >= total_items when the queue is exhausted).
template <bool EXPO, bool BRIDGE, class Dens, class Keys>
__device__ __forceinline__ unsigned long long run_stream(const MeshDev& M, const Dens& dens,
                                                         const Keys& philox,
                                                         unsigned long long first,
                                                         const McArgs& a, WarpAcc& W, int lane)
{
    const int n = M.n;
    const double invd = 1.0 / (double)(n - 1);
    const float invf = (float)invd;
    const uint32_t kmax = M.max_steps;
    const unsigned long long mesh_end = M.item_begin + (unsigned long long)M.n_nodes * M.chunks_per_node;

    if (lane == 0) {
#pragma unroll
        for (int s = 0; s < N_SETS; ++s) W.set_live[s] = 0u;
        W.used = 0u;
        W.cur = -1;
        W.cur_cursor = W.cur_end = W.cur_node = 0u;
        W.held = first;
        W.held_valid = 1;
        W.pending = 0ull;
        W.have_pending = 0;
    }
    __syncwarp();

    const float c4dt = (float)(-4.0 * M.dt * 0.69314718055994530942);
    constexpr bool bridge = BRIDGE;          // the kernel with the test inlines it
    // bridge cut for FP32 uniforms (no U >= 2^-24 lies below exp(-16.7))
    const float inv_dt = (float)(1.0 / M.dt), qmax = (float)(16.7 * M.dt);
    const float dth = (float)std::sqrt(16.7 * M.dt);
    constexpr float LN2F = 0.69314718055994530942f;
    float xs = 0.f, xt = 0.f;
    uint32_t k = 0, path = 0, node = 0, nid = 0;
    int set = 0;
    bool active = false;
    // single-mesh kernels of the lighter densities draw each step pair's
    // Philox block one pair ahead (the batch kernels, with their keys in
    // registers, and the 3- and 6-bump kernels run short of registers)
    constexpr bool kPipe = SDD_PIPELINE_RNG && Dens::kLight &&
                           std::is_same<Keys, ParamKeys>::value;
    uint4 rn = make_uint4(0u, 0u, 0u, 0u);     // Philox block of the coming step pair

    // `need` is warp-uniform: the refill runs once at the start and then only
    // after some path ended (only an ended path can free a lane, close a set or
    // change what can be handed out).  With exponential steps paths start only
    // on even pair iterations `it`, so every lane of the warp is at the same
    // place in its four-step block of lengths: the block's Philox call is
    // warp-uniform, once per two pairs (an ended lane may idle for a pair).
    unsigned dm = 0u;
    bool need = true;
    uint32_t it = 0;
    uint32_t hz = 0u, hw = 0u;                 // words z, w of the current length block
    for (int guard = 0;;) {
        if (need && (!EXPO || (it & 1u) == 0u)) {
            need = false;
            const unsigned idle = __ballot_sync(FULL, !active);
            constexpr bool kInlineRefill = !BRIDGE && std::is_same<Keys, ParamKeys>::value;
            const Refill rf = kInlineRefill ? stream_refill_inl(M, a, W, lane, dm, idle, mesh_end)
                                            : stream_refill(M, a, W, lane, dm, idle, mesh_end);
            dm = 0u;
            if ((rf.given >> lane) & 1u) {
                path = rf.path;
                node = rf.node;
                nid = M.node_ids ? M.node_ids[node] : node;
                set = rf.set;
                const int2 ij = M.nodes[node];
                xs = (float)ij.x * invf;
                xt = (float)ij.y * invf;
                k = 0;
                active = true;
                if constexpr (kPipe) rn = philox(make_uint4(0u, path, nid, 0u));
            }
            if (!__any_sync(FULL, active)) {
                // nothing running: this mesh is done once every set is written out
                if (W.have_pending && W.used == 0u) return W.pending;
                if (++guard > 64) return a.total_items;    // cannot happen; never spin
                need = true;
                continue;
            }
        }
        bool ended = false;
        if (active) {
            // two Euler-Maruyama steps from one Philox block, both computed
            // before the exit tests (a step after an exit is discarded)
            uint4 r;
            if constexpr (kPipe) {
                // this pair's block was drawn one pair ahead; draw the next one
                // now, in the same straight-line code as this pair's steps
                r = rn;
                rn = philox(make_uint4((k >> 1) + 1u, path, nid, 0u));
            } else {
                r = philox(make_uint4(k >> 1, path, nid, 0u));
            }
            // fa, fb: the steps' lengths over dt (1, or E = -ln U when the
            // steps are exponential)
            float fa = 1.0f, fb = 1.0f;
            if constexpr (EXPO) {
                uint32_t wa = hz, wb = hw;
                if ((it & 1u) == 0u) {                 // k = 4q: a new block of four lengths
                    const uint4 L = philox(make_uint4(k >> 2, path, nid, 2u));
                    wa = L.x;
                    wb = L.y;
                    hz = L.z;
                    hw = L.w;
                }
                fa = exp_unit_log2_f32(wa) * LN2F;
                fb = exp_unit_log2_f32(wb) * LN2F;
            }
            float na, ca, sa, nb, cb, sb;
            box_muller_f32_step(r.x, r.y, c4dt * fa, na, ca, sa);
            box_muller_f32_step(r.z, r.w, c4dt * fb, nb, cb, sb);
            float as, at;
            dens.advance(xs, xt, as, at, fa);
            const float y1s = fmaf(na, ca, as), y1t = fmaf(na, sa, at);
            dens.advance(y1s, y1t, as, at, fb);
            const float y2s = fmaf(nb, cb, as), y2t = fmaf(nb, sb, at);
            // one test for both steps: every coordinate inside (0,1), and, with
            // the bridge test, every coordinate of x, y1, y2 farther than
            // sqrt(qmax) from the sides (no crossing probability to draw)?
            const float lo = fminf(fminf(y1s, y1t), fminf(y2s, y2t));
            const float hi = fmaxf(fmaxf(y1s, y1t), fmaxf(y2s, y2t));
            bool fast = (lo > 0.f) & (hi < 1.f) & (k + 2u < kmax);
            if (bridge) {
                float d = dth;
                if constexpr (EXPO) d = sqrt_approx(qmax * fmaxf(fa, fb));
                fast = fast & (fminf(lo, fminf(xs, xt)) >= d) & (fmaxf(hi, fmaxf(xs, xt)) <= 1.f - d);
            }
            if (fast) {
                xs = y2s;
                xt = y2t;
                k += 2u;
            } else {
                // exit, bridge crossing or step cap within this pair (rare)
                float ps = xs, pt = xt, qs = y1s, qt = y1t;   // the step that ended
                float tau = 0.f;
                bool capped = false, dummy = false;
                int e = -1;
                k += 1u;
                const bool out1 = (y1s <= 0.f) | (y1s >= 1.f) | (y1t <= 0.f) | (y1t >= 1.f);
                if (out1) {
                    e = exit_edge<float>(xs, xt, y1s, y1t, tau);
                } else if (bridge && (e = bridge_exit_inl<float>(xs, xt, y1s, y1t,
                                                              EXPO ? inv_dt / fa : inv_dt,
                                                              EXPO ? qmax * fa : qmax, philox,
                                                              k - 1u, path, nid, tau, dummy)) >= 0) {
                } else if (k >= kmax) {
                    capped = true;
                } else {
                    ps = y1s; pt = y1t; qs = y2s; qt = y2t;
                    k += 1u;
                    const bool out2 = (y2s <= 0.f) | (y2s >= 1.f) | (y2t <= 0.f) | (y2t >= 1.f);
                    if (out2) {
                        e = exit_edge<float>(y1s, y1t, y2s, y2t, tau);
                    } else if (bridge && (e = bridge_exit_inl<float>(y1s, y1t, y2s, y2t,
                                                                  EXPO ? inv_dt / fb : inv_dt,
                                                                  EXPO ? qmax * fb : qmax,
                                                                  philox, k - 1u, path, nid, tau,
                                                                  dummy)) >= 0) {
                    } else if (k >= kmax) {
                        capped = true;
                    }
                }
                if (e >= 0 || capped) {
                    if (e < 0) e = nearest_edge<float>(qs, qt, tau);
                    const int2 ij = M.nodes[node];
                    const double td = (double)tau;
                    const double d0 = lookup(M.edges + (size_t)e * n, n, td) - (double)ij.x * invd;
                    const double d1 = lookup(M.edges + (size_t)(4 + e) * n, n, td) - (double)ij.y * invd;
                    atomicAdd(&W.s[set][0], (unsigned long long)__double2ll_rn(d0 * FX_SCALE));
                    atomicAdd(&W.s[set][1], (unsigned long long)__double2ll_rn(d1 * FX_SCALE));
                    atomicAdd(&W.q[set][0], (unsigned long long)__double2ll_rn(d0 * d0 * FX_SCALE));
                    atomicAdd(&W.q[set][1], (unsigned long long)__double2ll_rn(d1 * d1 * FX_SCALE));
                    atomicAdd(&W.steps[set], (unsigned long long)k);
                    atomicAdd(&W.caps[set], capped ? 1u : 0u);
                    atomicAdd(&W.paths[set], 1u);
                    active = false;
                    ended = true;
                } else {
                    xs = y2s;                       // both steps stayed inside
                    xt = y2t;
                }
                (void)ps; (void)pt;
            }
        }
        dm |= __ballot_sync(FULL, ended);          // kept until the next refill
        need = dm != 0u;
        ++it;
    }
}

// Density class of a mesh: a compile-time index for the FP32 path kernel, so
// each family gets a kernel (and a register allocation) of its own.
enum FamClass { FC_RING = 0, FC_RIDGE, FC_BUMPS1, FC_BUMPS2, FC_BUMPS3, FC_BUMPS6, FC_TABLE, FC_ANY };

__host__ __device__ __forceinline__ int fam_class(int family, int nb)
{
    if (family == SDD_FAMILY_RING) return FC_RING;
    if (family == SDD_FAMILY_RIDGE) return FC_RIDGE;
    if (family == SDD_FAMILY_TABLE) return FC_TABLE;
    if (nb <= 1) return FC_BUMPS1;
    if (nb == 2) return FC_BUMPS2;
    if (nb == 3) return FC_BUMPS3;
    return FC_BUMPS6;
}

template <int FC, bool EXPO, bool BRIDGE, class Keys>
__device__ __forceinline__ unsigned long long stream_fc(const MeshDev& M, const Keys& keys,
                                                        unsigned long long item, const McArgs& a,
                                                        WarpAcc& W, int lane)
{
    if constexpr (FC == FC_RING) { RingF32 d; d.load(M); return run_stream<EXPO, BRIDGE>(M, d, keys, item, a, W, lane); }
    if constexpr (FC == FC_RIDGE) { RidgeF32 d; d.load(M); return run_stream<EXPO, BRIDGE>(M, d, keys, item, a, W, lane); }
    if constexpr (FC == FC_TABLE) { TableF32 d; d.load(M); return run_stream<EXPO, BRIDGE>(M, d, keys, item, a, W, lane); }
    if constexpr (FC == FC_BUMPS1) { BumpsF32<1> d; d.load(M); return run_stream<EXPO, BRIDGE>(M, d, keys, item, a, W, lane); }
    if constexpr (FC == FC_BUMPS2) { BumpsF32<2> d; d.load(M); return run_stream<EXPO, BRIDGE>(M, d, keys, item, a, W, lane); }
    if constexpr (FC == FC_BUMPS3) { BumpsF32<3> d; d.load(M); return run_stream<EXPO, BRIDGE>(M, d, keys, item, a, W, lane); }
    if constexpr (FC == FC_BUMPS6) {
        BumpsF32<SDD_MAX_BUMPS> d;
        d.load(M);
        return run_stream<EXPO, BRIDGE>(M, d, keys, item, a, W, lane);
    }
    return a.total_items;
}

template <int FC, bool EXPO, bool BRIDGE, class Keys>
__device__ __forceinline__ unsigned long long dispatch_stream(const MeshDev& M, const Keys& keys,
                                                              unsigned long long item,
                                                              const McArgs& a, WarpAcc& W, int lane)
{
    if constexpr (FC != FC_ANY) {
        return stream_fc<FC, EXPO, BRIDGE>(M, keys, item, a, W, lane);
    } else {
        switch (fam_class(M.family, M.nb)) {
            case FC_RING: return stream_fc<FC_RING, EXPO, BRIDGE>(M, keys, item, a, W, lane);
            case FC_RIDGE: return stream_fc<FC_RIDGE, EXPO, BRIDGE>(M, keys, item, a, W, lane);
            case FC_TABLE: return stream_fc<FC_TABLE, EXPO, BRIDGE>(M, keys, item, a, W, lane);
            case FC_BUMPS1: return stream_fc<FC_BUMPS1, EXPO, BRIDGE>(M, keys, item, a, W, lane);
            case FC_BUMPS2: return stream_fc<FC_BUMPS2, EXPO, BRIDGE>(M, keys, item, a, W, lane);
            case FC_BUMPS3: return stream_fc<FC_BUMPS3, EXPO, BRIDGE>(M, keys, item, a, W, lane);
            default: return stream_fc<FC_BUMPS6, EXPO, BRIDGE>(M, keys, item, a, W, lane);
        }
    }
}

// ------------------------------------------------------ path kernel ----
// Mesh record of a work item: batched launches binary-search the per-mesh
// item offsets; single-mesh launches read the record passed by value, staged
// in shared memory by the block.
__device__ __forceinline__ int find_mesh(const uint64_t* __restrict__ off, int n_meshes, uint64_t x)
{
    int lo = 0, hi = n_meshes;                 // off[lo] <= x < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// ONE: single-mesh launch (record and round keys from the kernel parameters);
// otherwise a batch (records in global memory, one key per mesh).  FC: the
// density class the FP32 kernel is specialised for (FC_ANY: every class).
// EXPO: FP32 kernel with exponential time stepping (FP64 stepping reads the
// stepper from the mesh record).
// Launch shape of a path kernel: blocks of 128 threads for the narrow
// kernels (8 per SM, 7 with the bridge test), else MC_THREADS threads (the
// launcher asks path_threads; the grid is the occupancy API's count x SMs).
__host__ __device__ constexpr bool narrow_kernel(int prec, bool one, int fc, bool expo)
{
    return prec == SDD_FP32_STEP && one && !expo &&
           (fc == FC_RING || fc == FC_RIDGE || fc == FC_TABLE);
}

template <int PREC, bool ONE, int FC, bool EXPO, bool BRIDGE>
struct PathShape {
    static constexpr bool kNarrow = narrow_kernel(PREC, ONE, FC, EXPO);
    static constexpr int threads = kNarrow ? 128 : MC_THREADS;
    static constexpr int min_blocks = PREC == SDD_FP64 ? SDD_MC_MIN_BLOCKS_F64
                                      : kNarrow ? (BRIDGE ? 7 : 8) : SDD_MC_MIN_BLOCKS_F32;
};

template <int PREC, bool ONE, int FC, bool EXPO = false, bool BRIDGE = false>
__global__ void __launch_bounds__(PathShape<PREC, ONE, FC, EXPO, BRIDGE>::threads,
                                  PathShape<PREC, ONE, FC, EXPO, BRIDGE>::min_blocks)
k_paths(const __grid_constant__ McArgs a)
{
    __shared__ MeshDev single;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    if constexpr (ONE) {
        const int* src = reinterpret_cast<const int*>(&a.single);
        int* dst = reinterpret_cast<int*>(&single);
        for (int q = tid; q < (int)(sizeof(MeshDev) / sizeof(int)); q += blockDim.x) dst[q] = src[q];
        __syncthreads();
    }
    if constexpr (PREC == SDD_FP64) {
        // FP64 stepping: one item at a time, compensated FP64 lane sums
        __shared__ AccSmem acc;
        for (;;) {
            unsigned long long item = 0;
            if (lane == 0) item = a.item_base + atomicAdd(a.queue, 1ull);
            item = __shfl_sync(FULL, item, 0);
            if (item >= a.total_items) return;
            const MeshDev& M = ONE ? single : a.meshes[find_mesh(a.item_off, a.n_meshes, item)];
            const uint64_t local = item - M.item_begin;
            const uint32_t node = (uint32_t)(local / M.chunks_per_node);
            const uint32_t chunk = (uint32_t)(local % M.chunks_per_node);
            if (chunk < M.chunk_begin) continue;       // summed by the run this one continues
            Slot* out = a.slots + item;
            if constexpr (ONE) {
                const ParamKeys keys{a.rk};
                dispatch<PREC>(M, keys, node, chunk, out, acc, tid, lane);
            } else {
                const RegKeys keys{M.key0, M.key1};
                dispatch<PREC>(M, keys, node, chunk, out, acc, tid, lane);
            }
        }
    } else {
        // FP32 stepping: path streams across the items of a mesh
        constexpr int kWarps = PathShape<PREC, ONE, FC, EXPO, BRIDGE>::threads / 32;
        __shared__ WarpAcc wacc[kWarps];
        __shared__ uint32_t wkeys[kWarps][20];            // batch: round keys per warp
        (void)wkeys;                                      // (single mesh: kernel parameters)
        WarpAcc& W = wacc[tid >> 5];
        unsigned long long item = 0;
        if (lane == 0) item = a.item_base + atomicAdd(a.queue, 1ull);
        item = __shfl_sync(FULL, item, 0);
        while (item < a.total_items) {
            const MeshDev& M = ONE ? single : a.meshes[find_mesh(a.item_off, a.n_meshes, item)];
            if constexpr (ONE) {
                const ParamKeys keys{a.rk};
                item = dispatch_stream<FC, EXPO, BRIDGE>(M, keys, item, a, W, lane);
            } else {
                __syncwarp();
                if (lane < 20) {
                    const uint32_t r = (uint32_t)(lane >> 1);
                    wkeys[tid >> 5][lane] = (lane & 1) ? M.key1 + r * 0xBB67AE85u
                                                       : M.key0 + r * 0x9E3779B9u;
                }
                __syncwarp();
                const SmemKeys keys{wkeys[tid >> 5]};
                item = dispatch_stream<FC, EXPO, BRIDGE>(M, keys, item, a, W, lane);
            }
        }
    }
}

// ---------------------------------------------- per-node reduction ----
// One thread per node: the node's chunk slots are combined in chunk order
// (compensated), then mean = X0 + S/N and stderr = sqrt((Q - S^2/N)/(N(N-1)))
// (§2.2), and the mesh's counters are accumulated (integer atomics and an
// atomic max of the non-negative stderr bit pattern: order-independent).
__global__ void __launch_bounds__(256) k_reduce(const __grid_constant__ McArgs a)
{
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.total_nodes) return;
    int m = 0;
    if (a.meshes != nullptr) m = find_mesh(a.node_off, a.n_meshes, g);
    const MeshDev& M = a.meshes != nullptr ? a.meshes[m] : a.single;
    const uint64_t v = g - M.node_begin;
    const uint64_t base = M.item_begin + v * M.chunks_per_node;
    double sh[2] = {0, 0}, sl[2] = {0, 0}, qh[2] = {0, 0}, ql[2] = {0, 0};
    double st[2] = {0, 0}, qt[2] = {0, 0};
    unsigned long long ties = 0, caps = 0, steps = 0;
    unsigned long long paths = 0;
    const bool fixed = M.precision == SDD_FP32_STEP;
    for (uint32_t c = 0; c < M.chunks_per_node; ++c) {
        const Slot& S = a.slots[base + c];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (fixed) {
                // exact: |fx| < 2^53
                two_sum_add(sh[q], sl[q], (double)S.fx_s[q] * (1.0 / FX_SCALE));
                two_sum_add(qh[q], ql[q], (double)S.fx_q[q] * (1.0 / FX_SCALE));
            } else {
                sl[q] += S.s_lo[q];
                two_sum_add(sh[q], sl[q], S.s_hi[q]);
                ql[q] += S.q_lo[q];
                two_sum_add(qh[q], ql[q], S.q_hi[q]);
                st[q] += S.st[q];
                qt[q] += S.qt[q];
            }
        }
        ties += S.ties;
        caps += S.caps;
        steps += S.steps;
        paths += S.paths;
    }
    const double N = (double)M.paths;
    const int2 ij = M.nodes[v];
    const uint64_t vo = M.node_ids ? (uint64_t)M.node_ids[v] : v;   // output row
    const double x0[2] = {(double)ij.x / (double)(M.n - 1), (double)ij.y / (double)(M.n - 1)};
    sdd_node_sums out;
    double se_max = 0.0;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const double snt = sh[q] + sl[q];
        const double qnt = qh[q] + ql[q];
        out.sum_nt[q] = snt;
        out.sumsq_nt[q] = qnt;
        out.sum[q] = snt + st[q];
        out.sumsq[q] = qnt + qt[q];
        const double S = out.sum[q], Q = out.sumsq[q];
        const double var = fmax(Q - S * S / N, 0.0) / (N * (N - 1.0));
        const double se = sqrt(var);
        se_max = fmax(se_max, se);
        if (M.mean) M.mean[2 * vo + q] = x0[q] + S / N;
        if (M.stderr_) M.stderr_[2 * vo + q] = se;
    }
    out.paths = paths;
    out.ties = ties;
    out.non_exits = caps;
    out.steps = steps;
    if (M.sums) M.sums[vo] = out;
    atomicAdd(&M.stats->steps, steps);
    atomicAdd(&M.stats->ties, ties);
    atomicAdd(&M.stats->caps, caps);
    if (paths != (unsigned long long)M.paths) atomicAdd(&M.stats->lost, 1ull);
    atomicMax(&M.stats->max_stderr_bits, (unsigned long long)__double_as_longlong(se_max));
}

// Few-point interface: interpolated nodes from the Monte Carlo nodes (or the
// boundary map) at both ends of their stretch of interface line.
__global__ void k_interp(const InterpEntry* __restrict__ e, int64_t count)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= count) return;
    const InterpEntry E = e[g];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const double A = E.a >= 0 ? E.mean[2 * E.a + c] : E.ca[c];
        const double B = E.b >= 0 ? E.mean[2 * E.b + c] : E.cb[c];
        E.mean[2 * E.q + c] = (1.0 - E.w) * A + E.w * B;
        if (E.se) {
            const double sa = E.a >= 0 ? E.se[2 * E.a + c] : 0.0;
            const double sb = E.b >= 0 ? E.se[2 * E.b + c] : 0.0;
            E.se[2 * E.q + c] = (1.0 - E.w) * sa + E.w * sb;
        }
    }
}

}  // namespace

int launch_interp(const InterpEntry* d_entries, int64_t count, cudaStream_t stream)
{
    if (count <= 0) return SDD_OK;
    k_interp<<<(unsigned)((count + 255) / 256), 256, 0, stream>>>(d_entries, count);
    SDD_CUDA(cudaGetLastError());
    count_launch();
    return SDD_OK;
}

// ------------------------------------------------------------ host side ----
void fill_fp32_params(MeshDev& m, const sdd_density& d)
{
    const double LOG2E = 1.44269504088896340736;
    for (int q = 0; q < 48; ++q) m.pf[q] = 0.0f;
    for (int q = 0; q < 32; ++q) m.pd[q] = q < d.n_params ? d.params[q] : 0.0;
    m.sgn = d.coef_mode == SDD_COEF_INV_W ? -1.0 : 1.0;
    if (d.family == SDD_FAMILY_BUMPS) {
        const int nb = (int)d.params[0];
        m.nb = nb;
        for (int b = 0; b < nb; ++b) {
            const double* q = d.params + 1 + 5 * b;
            m.pf[8 * b + 0] = (float)q[0];
            m.pf[8 * b + 1] = (float)q[1];
            m.pf[8 * b + 2] = (float)q[2];
            m.pf[8 * b + 3] = (float)(q[3] * LOG2E);
            m.pf[8 * b + 4] = (float)(q[4] * LOG2E);
            m.pf[8 * b + 5] = (float)(-2.0 * q[3]);
            m.pf[8 * b + 6] = (float)(-2.0 * q[4]);
        }
    } else if (d.family == SDD_FAMILY_RING) {
        const double A = d.params[0], cs = d.params[1], ct = d.params[2], k = d.params[3],
                     r0 = d.params[4];
        m.nb = 0;
        m.pf[0] = (float)cs;
        m.pf[1] = (float)ct;
        m.pf[2] = (float)r0;
        m.pf[3] = (float)(-2.0 * k * LOG2E);
        m.pf[4] = (float)(4.0 * A);
        m.pf[5] = (float)(m.sgn * -8.0 * A * k);
        // u = k (r - r0): the kernel forms r - r0 and folds k into c1 and K
    } else if (d.family == SDD_FAMILY_TABLE) {
        m.nb = 0;                                // the table itself is passed by pointer
    } else {
        const double A = d.params[0], k = d.params[1], t0 = d.params[2], a = d.params[3],
                     f = d.params[4];
        m.nb = 0;
        m.pf[0] = (float)A;
        m.pf[1] = (float)(k * LOG2E);
        m.pf[2] = (float)t0;
        m.pf[3] = (float)a;
        m.pf[4] = (float)f;
        m.pf[5] = (float)(-2.0 * k);
        m.pf[6] = (float)(-2.0 * 3.14159265358979323846 * a * f);
    }
}

// Kernel of a launch: precision, single mesh or batch, kernel class (density
// class + KC_EXPO for exponential time stepping + KC_BRIDGE for the
// Brownian-bridge test).
using PathKernel = void (*)(McArgs);

template <bool EXPO, bool BRIDGE>
static PathKernel path_kernel_fp32(bool one, int fc)
{
    if (!one) {
        switch (fc) {
            case FC_RING: return k_paths<SDD_FP32_STEP, false, FC_RING, EXPO, BRIDGE>;
            case FC_RIDGE: return k_paths<SDD_FP32_STEP, false, FC_RIDGE, EXPO, BRIDGE>;
            case FC_TABLE: return k_paths<SDD_FP32_STEP, false, FC_TABLE, EXPO, BRIDGE>;
            case FC_BUMPS1: return k_paths<SDD_FP32_STEP, false, FC_BUMPS1, EXPO, BRIDGE>;
            case FC_BUMPS2: return k_paths<SDD_FP32_STEP, false, FC_BUMPS2, EXPO, BRIDGE>;
            case FC_BUMPS3: return k_paths<SDD_FP32_STEP, false, FC_BUMPS3, EXPO, BRIDGE>;
            case FC_BUMPS6: return k_paths<SDD_FP32_STEP, false, FC_BUMPS6, EXPO, BRIDGE>;
            default: return k_paths<SDD_FP32_STEP, false, FC_ANY, EXPO, BRIDGE>;
        }
    }
    switch (fc) {
        case FC_RING: return k_paths<SDD_FP32_STEP, true, FC_RING, EXPO, BRIDGE>;
        case FC_RIDGE: return k_paths<SDD_FP32_STEP, true, FC_RIDGE, EXPO, BRIDGE>;
        case FC_TABLE: return k_paths<SDD_FP32_STEP, true, FC_TABLE, EXPO, BRIDGE>;
        case FC_BUMPS1: return k_paths<SDD_FP32_STEP, true, FC_BUMPS1, EXPO, BRIDGE>;
        case FC_BUMPS2: return k_paths<SDD_FP32_STEP, true, FC_BUMPS2, EXPO, BRIDGE>;
        case FC_BUMPS3: return k_paths<SDD_FP32_STEP, true, FC_BUMPS3, EXPO, BRIDGE>;
        default: return k_paths<SDD_FP32_STEP, true, FC_BUMPS6, EXPO, BRIDGE>;
    }
}

// Threads per block of that kernel (PathShape).
static int path_threads(int precision, bool one, int kc)
{
    const bool expo = precision != SDD_FP64 && (kc & KC_EXPO) != 0;
    const int fc = precision == SDD_FP64 ? (int)FC_ANY : (kc & (KC_EXPO - 1));
    return narrow_kernel(precision, one, fc, expo) ? 128 : MC_THREADS;
}

static PathKernel path_kernel(int precision, bool one, int kc)
{
    if (precision == SDD_FP64) return one ? k_paths<SDD_FP64, true, FC_ANY> : k_paths<SDD_FP64, false, FC_ANY>;
    const int fc = kc & (KC_EXPO - 1);
    const bool bridge = (kc & KC_BRIDGE) != 0;
    if (kc & KC_EXPO) return bridge ? path_kernel_fp32<true, true>(one, fc) : path_kernel_fp32<true, false>(one, fc);
    return bridge ? path_kernel_fp32<false, true>(one, fc) : path_kernel_fp32<false, false>(one, fc);
}

int mesh_kernel_class(int family, int nb, int stepper, int exit_test)
{
    return fam_class(family, nb) + (stepper == SDD_STEP_EXPONENTIAL ? KC_EXPO : 0) +
           (exit_test == SDD_EXIT_BRIDGE ? KC_BRIDGE : 0);
}

int mc_grid_blocks(int precision, int kc, bool one, int* blocks, int* threads)
{
    int dev = 0, sms = 0, per_sm = 0;
    SDD_CUDA(cudaGetDevice(&dev));
    SDD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SDD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, reinterpret_cast<const void*>(path_kernel(precision, one, kc)),
        path_threads(precision, one, kc), 0));
    *blocks = sms * std::max(per_sm, 1);
    if (threads) *threads = path_threads(precision, one, kc);
    return SDD_OK;
}

int launch_mc(const McArgs& args, int precision, int kc, cudaStream_t stream)
{
    if (args.total_items <= args.item_base) return SDD_OK;
    const bool one = args.meshes == nullptr;
    int blocks = 0, threads = 0;
    int rc = mc_grid_blocks(precision, kc, one, &blocks, &threads);
    if (rc) return rc;
    return launch_mc_sized(args, precision, kc, blocks, stream);
}

static int launch_paths_sized(const McArgs& args, int precision, int kc, int blocks,
                              cudaStream_t stream)
{
    if (args.total_items <= args.item_base) return SDD_OK;
    const bool one = args.meshes == nullptr;
    const int threads = path_threads(precision, one, kc);
    const uint64_t max_blocks = ((args.total_items - args.item_base) * 32 + threads - 1) / threads;
    if ((uint64_t)blocks > max_blocks) blocks = (int)max_blocks;
    if (blocks < 1) blocks = 1;
    SDD_CUDA(cudaMemsetAsync(args.queue, 0, sizeof(unsigned long long), stream));
    path_kernel(precision, one, kc)<<<blocks, threads, 0, stream>>>(args);
    SDD_CUDA(cudaGetLastError());
    count_launch();
    return SDD_OK;
}

int launch_mc_reduce(const McArgs& args, cudaStream_t stream)
{
    if (args.total_nodes == 0) return SDD_OK;
    const unsigned rb = (unsigned)((args.total_nodes + 255) / 256);
    k_reduce<<<rb, 256, 0, stream>>>(args);
    SDD_CUDA(cudaGetLastError());
    count_launch();
    return SDD_OK;
}

int launch_mc_paths(const McArgs& args, int precision, int kc, cudaStream_t stream)
{
    if (args.total_items <= args.item_base) return SDD_OK;
    int blocks = 0;
    int rc = mc_grid_blocks(precision, kc, args.meshes == nullptr, &blocks, nullptr);
    if (rc) return rc;
    return launch_paths_sized(args, precision, kc, blocks, stream);
}

int launch_mc_sized(const McArgs& args, int precision, int kc, int blocks, cudaStream_t stream)
{
    if (args.total_items <= args.item_base) return SDD_OK;
    int rc = launch_paths_sized(args, precision, kc, blocks, stream);
    if (rc) return rc;
    return launch_mc_reduce(args, stream);
}

}  // namespace sdd
