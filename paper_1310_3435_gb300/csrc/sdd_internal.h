// Internal declarations shared by the translation units of libsdd.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "sdd.h"

namespace sdd {

// ---------------------------------------------------------------- errors --
void set_error(const std::string& msg);
void clear_error();
int fail(int code, const std::string& msg);
// Records a CUDA error (if any) and returns SDD_ERR_CUDA, else SDD_OK.
int cuda_status(cudaError_t e, const char* what);
void count_launch(uint64_t k = 1);       // kernels launched (wraps modulo 2^64)
uint64_t launches_now();

#define SDD_CUDA(call)                                                  \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return ::sdd::cuda_status(e_, #call);    \
    } while (0)

// --------------------------------------------------- per-mesh MC record --
// One record per mesh in a Monte Carlo launch.  Parameters are read by the
// path kernel at the start of each work item (warp-uniform loads).
struct McStatsDev {
    unsigned long long steps;
    unsigned long long ties;
    unsigned long long caps;
    unsigned long long max_stderr_bits;   // bit pattern of a non-negative double
    unsigned long long lost;              // nodes whose path count differs from N (0)
};

struct MeshDev {
    int32_t n;              // grid points per side
    int32_t family;         // SDD_FAMILY_*
    int32_t nb;             // bumps (BUMPS family)
    int32_t precision;      // SDD_FP64 | SDD_FP32_STEP
    uint32_t key0, key1;    // Philox key = seed (lo, hi)
    uint32_t paths;         // N per node
    uint32_t chunk;         // paths per work item
    uint32_t chunks_per_node;
    uint32_t max_steps;     // step cap per path (< 2^32)
    int32_t bridge;         // 1: Brownian-bridge exit test after each step
    int32_t stepper;        // SDD_STEP_EULER | SDD_STEP_EXPONENTIAL
    int64_t n_nodes;
    uint64_t item_begin;    // first work item of this mesh
    uint64_t node_begin;    // first global node of this mesh
    double dt;
    double sqrt2dt;
    double tie_delta;
    double sgn;             // +1: c = w, -1: c = 1/w
    const int2* nodes;      // [n_nodes] (i, j) of the nodes the Monte Carlo runs on
    const uint32_t* node_ids;  // their index in the plan's interface list (Philox
                               // counter word, output row); NULL: the position itself
    const double* edges;    // [2][4][n]
    sdd_node_sums* sums;    // [n_nodes] out
    double* mean;           // [n_nodes][2] out (may be null)
    double* stderr_;        // [n_nodes][2] out (may be null)
    McStatsDev* stats;      // out
    float pf[48];           // FP32-stepping parameters, pre-transformed per family
    double pd[32];          // raw parameters (FP64 stepping)
    const double* tab64;    // TABLE family: [tn][tn] ln w (FP64 stepping)
    const float4* cell32;   // FP32 stepping: per cell (c1, c2, c3, 0) with L = c0 + (c1 fa +
                            // c2 fb + c3 fa fb) / (tn-1) in the cell's local coordinates
    int32_t tn;
    uint32_t chunk_begin;   // items of a node with chunk index < chunk_begin hold the
                            // sums of the run this one continues: not run again
};

// Partial sums of one work item (one chunk of paths of one node).
struct Slot {
    double s_hi[2], s_lo[2];   // sum of d over non-tie paths (compensated pair)
    double q_hi[2], q_lo[2];   // sum of d^2 over non-tie paths
    double st[2], qt[2];       // sums over tie-flagged paths
    long long fx_s[2], fx_q[2];  // FP32 stepping: exact 2^-40 fixed-point sums of d, d^2
    uint32_t ties, caps;
    unsigned long long steps;
    uint32_t paths, reserved;  // paths accumulated (checked against N per node)
};

// Fills the family-specific FP32 parameter block of a mesh record.
void fill_fp32_params(MeshDev& m, const sdd_density& d);

// Arguments of a Monte Carlo launch.  Batched: `meshes` points to n_meshes
// device records and item_off / node_off to their device prefix sums
// (n_meshes + 1 entries).  Single mesh: meshes = NULL and `single` holds the
// record (item_begin = node_begin = 0).
struct McArgs {
    const MeshDev* meshes;
    int n_meshes;
    const uint64_t* item_off;
    const uint64_t* node_off;
    uint64_t total_items;        // work items [item_base, total_items) are run
    uint64_t total_nodes;
    uint64_t item_base;          // first work item of the launch (0 but in resumed runs)
    unsigned long long* queue;   // device work counter (reset by the launcher)
    Slot* slots;                 // total_items entries
    MeshDev single;
    uint32_t rk[20];             // single mesh: Philox round keys (k0, k1) of rounds 0..9
};

// Kernel class of a mesh for the FP32 path kernel: its density class (one
// kernel per class; kFamAny selects the kernel that handles every class) plus
// KC_EXPO for exponential time stepping and KC_BRIDGE for the Brownian-bridge
// exit test (kernels with the test inline it; the others leave it out).
// FP64 stepping has one kernel.
int mesh_kernel_class(int family, int nb, int stepper, int exit_test);
constexpr int kFamAny = 7;
constexpr int KC_EXPO = 8;
constexpr int KC_BRIDGE = 16;

// Interpolated interface node of a few-point interface (§3.6): value =
// (1 - w) A + w B per component, A / B the mean (and std-err) of interface
// node a / b, or the boundary-map constant ca / cb when a / b < 0.
struct InterpEntry {
    double* mean;           // [n_nodes][2] of the plan
    double* se;             // may be null
    int64_t q, a, b;
    double w;
    double ca[2], cb[2];
};
int launch_interp(const InterpEntry* d_entries, int64_t count, cudaStream_t stream);

// Mesh quality: cells' Q(K) (max, sum, folds) of `u` and of `ref`, l_inf of w.
struct QualityDev {
    unsigned long long q_max_bits, q_ref_max_bits;
    double q_sum, q_ref_sum;
    unsigned long long folds, ref_folds, l_inf_bits;
};
int launch_quality(int n, int family, const double* params, const double* tab, int tn,
                   const double* u, const double* ref, QualityDev* d_out, cudaStream_t stream);

// Perona-Malik smoothing of the mesh u [n][n][2] (device), `steps` FTCS steps
// ping-ponged with `scratch` (device, same size); the result ends in u.
// hold: null, or n bytes (device) marking held columns (bit 0) and rows
// (bit 1), whose nodes stay fixed like the boundary.
int launch_smooth(int n, double* u, double* scratch, int steps, double dt, double k,
                  const uint8_t* hold, cudaStream_t stream);

// Launches the path kernel (for kernel class `kc`) and the per-node
// reduction.
int launch_mc(const McArgs& args, int precision, int kc, cudaStream_t stream);

// Same with a precomputed persistent-grid size (no device queries: usable
// while a stream is being captured into a CUDA graph).
int launch_mc_sized(const McArgs& args, int precision, int kc, int blocks, cudaStream_t stream);

// The two halves of launch_mc, for runs split over several calls: the path
// kernel over work items [item_base, total_items), and the per-node reduction
// over every item of the run.
int launch_mc_paths(const McArgs& args, int precision, int kc, cudaStream_t stream);
int launch_mc_reduce(const McArgs& args, cudaStream_t stream);

// Persistent-grid size of the path kernel for the current device.
int mc_grid_blocks(int precision, int kc, bool one, int* blocks, int* threads);

// ------------------------------------------------------- solve records --
struct SolveMeshDev {
    int32_t n;
    int32_t solver;
    int32_t max_iter;
    int32_t reserved;
    double tol;
    double omega;
    double* u;              // [n][n][2] mesh (in/out, FP64)
    const double* cx;       // [n][n-1]  c at (i+1/2, j)
    const double* cy;       // [n-1][n]  c at (i, j+1/2)
    const float* cxf;       // FP32 copies
    const float* cyf;
    float* work;            // FP32 workspace, 11 floats per grid node (r p q x z: 2 each, 1/diag)
    float* mg;              // multigrid levels of the subdomains (SubDev::mg_off)
};

struct SubDev {
    int32_t mesh;           // index into the SolveMeshDev array
    int32_t i0, i1, j0, j1; // interior: i0 < i < i1, j0 < j < j1
    int32_t slot;           // index of its SubStat record
    int64_t mg_off;         // first float of its multigrid levels in the mesh's mg buffer
};

// ------------------------------------------------ multigrid hierarchy --
// Coarse levels of a subdomain's geometric multigrid, the preconditioner of
// the FP32 CG.  Level 0 is the subdomain's interior (nx x ny nodes); level
// l + 1 halves (floor) each side of level l that has at least 2 nodes, until
// a level holds at most MG_COARSEST nodes or cannot shrink.  A coarse level
// is stored with a ring of padding around its interior (pitch nx + 2): the
// 9 planes of its Galerkin stencil (float), then the planes x, b, t
// (float2), each plane `plane` floats (even, so float2 planes stay aligned).
constexpr int MG_MAX_LEVELS = 16;
constexpr int MG_COARSEST = 32;

struct MgShape {
    int levels;                        // coarse levels (0: none)
    int nx[MG_MAX_LEVELS], ny[MG_MAX_LEVELS];   // [0]: the interior
    int cx[MG_MAX_LEVELS], cy[MG_MAX_LEVELS];   // level l was coarsened in x / in y
    int plane[MG_MAX_LEVELS];          // floats per plane of level l (l >= 1)
    int64_t off[MG_MAX_LEVELS];        // first float of level l (l >= 1)
    int64_t total;                     // floats of all coarse levels
};

__host__ __device__ inline void mg_shape(int nx, int ny, MgShape& s)
{
    s.levels = 0;
    s.total = 0;
    s.nx[0] = nx > 0 ? nx : 0;
    s.ny[0] = ny > 0 ? ny : 0;
    s.cx[0] = s.cy[0] = 0;
    s.plane[0] = 0;
    s.off[0] = 0;
    int l = 0;
    while (l + 1 < MG_MAX_LEVELS && s.nx[l] * s.ny[l] > MG_COARSEST) {
        const int cx = s.nx[l] >= 2, cy = s.ny[l] >= 2;
        if (!cx && !cy) break;
        ++l;
        s.nx[l] = cx ? s.nx[l - 1] / 2 : s.nx[l - 1];
        s.ny[l] = cy ? s.ny[l - 1] / 2 : s.ny[l - 1];
        s.cx[l] = cx;
        s.cy[l] = cy;
        const int a = (s.nx[l] + 2) * (s.ny[l] + 2);
        s.plane[l] = a + (a & 1);
        s.off[l] = s.total;
        s.total += 15 * (int64_t)s.plane[l];
    }
    s.levels = l;
}

struct SubStat {
    int32_t iterations;
    int32_t converged;
    double rel_residual;
};

// c at edge midpoints (FP64 and FP32 copies) for one mesh.
int launch_edge_coefs(int n, int family, int coef_mode, const double* params, const double* tab,
                      int tn, double* cx, double* cy, float* cxf, float* cyf, cudaStream_t stream);
// Boundary tables + interface values into the mesh, Coons-patch start values
// in the subdomain interiors.
int launch_fill_mesh(int n, const double* edges, const int2* nodes, int64_t n_nodes,
                     const double* iface, double* u, const SubDev* subs, int n_subs,
                     cudaStream_t stream);
// Arguments of a solve launch: batched (`meshes` = device records) or one mesh
// (`meshes` = NULL, record in `single`).  One CTA per entry of `subs`.
struct SolveArgs {
    const SolveMeshDev* meshes;
    SolveMeshDev single;
    const SubDev* subs;
    int n_subs;
    int solver_mask;            // bit 0: some subdomain uses SOR, bit 1: multigrid CG, bit 2: Jacobi CG
    int threads;                // CTA size: 256, 512 or 1024 (other: 1024)
    SubStat* stats;
};
int launch_solve(const SolveArgs& args, cudaStream_t stream);

// Batched Dirichlet fill: boundary tables and interface values of several
// meshes into their mesh arrays, one launch.  `off` holds the device prefix
// sums of the per-mesh element counts 4 n + n_nodes (n_meshes + 1 entries).
struct FillDev {
    int32_t n;
    int32_t reserved;
    int64_t n_nodes;
    const double* edges;
    const int2* nodes;
    const double* iface;
    double* u;
};
int launch_fill_batched(const FillDev* d_fill, const uint64_t* d_off, int n_meshes,
                        uint64_t total, cudaStream_t stream);

}  // namespace sdd

// ------------------------------------------------------------------ plan --
// Plan: the request description, its host tables and its resident device
// buffers (allocated lazily, kept across calls).
struct sdd_plan {
    int n = 0, sx = 0, sy = 0;
    int device = 0;
    sdd_density dens{};
    int bmap_mode = 0;
    std::vector<int> ix, iy;               // interface lines
    std::vector<int32_t> h_nodes;          // [n_nodes][2] (i, j)
    std::vector<double> h_edges;           // [2][4][n]
    std::vector<sdd::SubDev> h_subs;
    int64_t n_nodes = 0;

    int2* d_nodes = nullptr;
    double* d_edges = nullptr;
    std::vector<double> h_table;           // TABLE density: [tn][tn] ln w (dens.table points here)
    double* d_tab64 = nullptr;
    float4* d_cell32 = nullptr;            // FP32 per-cell gradient coefficients

    // Monte Carlo
    unsigned long long* d_queue = nullptr;
    sdd::Slot* d_slots = nullptr;
    uint64_t slots_cap = 0;
    sdd_node_sums* d_sums = nullptr;
    double* d_mean = nullptr;
    double* d_stderr = nullptr;
    sdd::McStatsDev* d_stats = nullptr;
    uint64_t last_paths = 0;
    bool have_mc = false;
    // a Monte Carlo run split over calls (sdd_interface_mc_advance / _finish)
    bool resume_active = false;
    sdd_mc_params resume_mc{};
    uint64_t resume_next = 0, resume_total = 0;
    cudaEvent_t mc_done = nullptr;         // recorded after each single-plan Monte Carlo call
    // the run whose work items d_slots holds (the last whole single-plan run),
    // which a later run may continue (sdd_mc_params.path_begin)
    bool items_valid = false;
    sdd_mc_params items_mc{};
    int64_t items_nodes = 0;               // nodes the run ran on (few-point aware)
    uint64_t items_run = 0;                // whole single-plan runs so far (identifies the items)

    // subdomain solves
    double* d_u = nullptr;
    double* d_cx = nullptr;
    double* d_cy = nullptr;
    float* d_cxf = nullptr;
    float* d_cyf = nullptr;
    float* d_work = nullptr;
    float* d_mg = nullptr;                 // multigrid levels of all subdomains
    int64_t mg_floats = 0;
    sdd::SubDev* d_subs = nullptr;
    sdd::SubStat* d_substats = nullptr;
    bool coefs_ready = false;

    // few-point interface: Monte Carlo on a subset, interpolation for the rest
    int place_mode = 0;
    std::vector<uint8_t> h_mask;           // [n_nodes] 1 = Monte Carlo node
    int64_t n_mc = 0;                      // nodes the Monte Carlo runs on
    int2* d_mc_nodes = nullptr;            // [n_mc]
    uint32_t* d_mc_ids = nullptr;          // [n_mc] index in the interface list
    std::vector<sdd::InterpEntry> h_interp;   // pointers filled per call
    sdd::InterpEntry* d_interp = nullptr;
    double* d_interp_mean = nullptr;       // outputs the device entries point at
    double* d_interp_se = nullptr;
    sdd::QualityDev* d_quality = nullptr;

    cudaStream_t last_stream = nullptr;
};

