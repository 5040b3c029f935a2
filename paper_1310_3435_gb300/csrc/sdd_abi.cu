// C ABI of libsdd.so: plans, interface Monte Carlo, subdomain solves and the
// combined mesh generation (Bihlo & Haynes, §2.1-2.2, §3.2, §3.5).
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <cstdio>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sdd_internal.h"

namespace sdd {

// NVTX range around an ABI call (host timeline; a profiler filters kernels by
// it, e.g. ncu --nvtx --nvtx-include "sdd_interface_mc/").
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------- errors --
namespace {
thread_local std::string g_error;
std::atomic<uint64_t> g_launches{0};
}  // namespace

void set_error(const std::string& msg) { g_error = msg; }
void clear_error() { g_error.clear(); }
int fail(int code, const std::string& msg)
{
    g_error = msg;
    return code;
}
int cuda_status(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return SDD_OK;
    g_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) return SDD_ERR_OOM;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return SDD_ERR_NO_DEVICE;
    return SDD_ERR_CUDA;
}
void count_launch(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
uint64_t launches_now() { return g_launches.load(std::memory_order_relaxed); }

namespace {

// Device (or managed) memory?  Anything else is host memory and is copied.
bool is_device_ptr(const void* p)
{
    if (p == nullptr) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device memory is stream-ordered (cudaMallocAsync / cudaFreeAsync from the
// device's default pool), so creating and destroying plans and batches never
// synchronises the device: work already queued on other streams keeps
// running.  Allocations go to the stream named by an AllocOn guard (the
// call's stream, or the library's set-up stream).
thread_local cudaStream_t t_alloc_stream = nullptr;

struct AllocOn {
    cudaStream_t prev;
    explicit AllocOn(cudaStream_t s) : prev(t_alloc_stream) { t_alloc_stream = s; }
    ~AllocOn() { t_alloc_stream = prev; }
};

// Library stream for set-up work (plan tables, batch records), one per
// device, non-blocking so that it never waits for the caller's streams.
cudaStream_t setup_stream()
{
    static std::mutex mu;
    static cudaStream_t streams[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!streams[dev]) cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking);
    return streams[dev];
}

template <typename T>
int dev_alloc(T** p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    SDD_CUDA(cudaMallocAsync(reinterpret_cast<void**>(p), count * sizeof(T), t_alloc_stream));
    return SDD_OK;
}

template <typename T>
void dev_free(T*& p, cudaStream_t s)
{
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
}

int64_t interior_nodes(const SubDev& d)
{
    return (int64_t)std::max(d.i1 - d.i0 - 1, 0) * std::max(d.j1 - d.j0 - 1, 0);
}

// Subdomains in decreasing interior size: one CTA each, the largest (the
// longest solves) are scheduled first, so they do not set the tail.
void sort_largest_first(std::vector<SubDev>& v)
{
    auto size = [](const SubDev& d) {
        return (int64_t)std::max(d.i1 - d.i0 - 1, 0) * std::max(d.j1 - d.j0 - 1, 0);
    };
    std::stable_sort(v.begin(), v.end(), [&](const SubDev& a, const SubDev& b) { return size(a) > size(b); });
}

// Interface lines of an s-way split of n points: I_k = round(k (n-1)/s),
// halves rounded up, exact integer arithmetic.
std::vector<int> interface_lines(int n, int s)
{
    std::vector<int> v;
    for (int k = 1; k < s; ++k) v.push_back((int)((2LL * k * (n - 1) + s) / (2LL * s)));
    return v;
}

// Host FP64 evaluation of c for the paper's 1D boundary forms (§3.2).
double host_coef(const sdd_density& d, double s, double t)
{
    const double* p = d.params;
    double w;
    if (d.family == SDD_FAMILY_TABLE) {
        const int tn = d.tn;
        const double* T = d.table;
        const double m = (double)(tn - 1);
        const double x = s * m, y = t * m;
        const int a = std::min(std::max((int)std::floor(x), 0), tn - 2);
        const int b = std::min(std::max((int)std::floor(y), 0), tn - 2);
        const double fa = x - (double)a, fb = y - (double)b;
        const double L00 = T[b * tn + a], L10 = T[b * tn + a + 1];
        const double L01 = T[(b + 1) * tn + a], L11 = T[(b + 1) * tn + a + 1];
        w = std::exp((1.0 - fb) * ((1.0 - fa) * L00 + fa * L10) +
                     fb * ((1.0 - fa) * L01 + fa * L11));
    } else if (d.family == SDD_FAMILY_RING) {
        const double ds = s - p[1], dtt = t - p[2];
        const double u = p[3] * (std::sqrt(ds * ds + dtt * dtt) - p[4]);
        const double e = std::exp(-2.0 * std::fabs(u));
        w = 1.0 + p[0] * 4.0 * e / ((1.0 + e) * (1.0 + e));
    } else if (d.family == SDD_FAMILY_RIDGE) {
        const double v = t - p[2] - p[3] * std::sin(2.0 * 3.14159265358979323846 * p[4] * s);
        w = 1.0 + p[0] * std::exp(-p[1] * v * v);
    } else {
        w = 1.0;
        const int nb = (int)p[0];
        for (int b = 0; b < nb; ++b) {
            const double* q = p + 1 + 5 * b;
            const double ds = s - q[1], dtt = t - q[2];
            w += q[0] * std::exp(-(q[3] * ds * ds + q[4] * dtt * dtt));
        }
    }
    return d.coef_mode == SDD_COEF_INV_W ? 1.0 / w : w;
}

int validate_density(const sdd_density* d)
{
    if (!d) return fail(SDD_ERR_INVALID_ARG, "density is NULL");
    if (d->coef_mode != SDD_COEF_W && d->coef_mode != SDD_COEF_INV_W)
        return fail(SDD_ERR_INVALID_ARG, "unknown coef_mode");
    if (d->n_params < 0 || d->n_params > SDD_MAX_PARAMS)
        return fail(SDD_ERR_INVALID_ARG, "n_params out of range");
    for (int q = 0; q < d->n_params; ++q)
        if (!std::isfinite(d->params[q])) return fail(SDD_ERR_INVALID_ARG, "non-finite parameter");
    if (d->family == SDD_FAMILY_BUMPS) {
        if (d->n_params < 1) return fail(SDD_ERR_INVALID_ARG, "BUMPS needs params[0] = nb");
        const double nbd = d->params[0];
        const int nb = (int)nbd;
        if (nbd != (double)nb || nb < 0 || nb > SDD_MAX_BUMPS)
            return fail(SDD_ERR_INVALID_ARG, "BUMPS: nb must be an integer in 0..6");
        if (d->n_params < 1 + 5 * nb) return fail(SDD_ERR_INVALID_ARG, "BUMPS: too few params");
        for (int b = 0; b < nb; ++b) {
            const double* q = d->params + 1 + 5 * b;
            if (q[3] < 0 || q[4] < 0) return fail(SDD_ERR_INVALID_ARG, "BUMPS: ks, kt must be >= 0");
            if (q[0] <= -1.0 / nb) return fail(SDD_ERR_INVALID_ARG, "BUMPS: w must stay positive");
        }
    } else if (d->family == SDD_FAMILY_TABLE) {
        if (d->tn < 2 || d->tn > SDD_MAX_TABLE)
            return fail(SDD_ERR_INVALID_ARG, "TABLE: tn must be in [2, SDD_MAX_TABLE]");
        if (!d->table) return fail(SDD_ERR_INVALID_ARG, "TABLE: table is NULL");
        for (int64_t q = 0; q < (int64_t)d->tn * d->tn; ++q)
            if (!std::isfinite(d->table[q]) || std::fabs(d->table[q]) > 700.0)
                return fail(SDD_ERR_INVALID_ARG, "TABLE: ln w must be finite, |ln w| <= 700");
    } else if (d->family == SDD_FAMILY_RING || d->family == SDD_FAMILY_RIDGE) {
        if (d->n_params < 5) return fail(SDD_ERR_INVALID_ARG, "RING/RIDGE need 5 params");
        if (d->params[0] <= -1.0) return fail(SDD_ERR_INVALID_ARG, "w must stay positive");
        if (d->family == SDD_FAMILY_RIDGE && d->params[1] < 0)
            return fail(SDD_ERR_INVALID_ARG, "RIDGE: k must be >= 0");
    } else {
        return fail(SDD_ERR_INVALID_ARG, "unknown density family");
    }
    return SDD_OK;
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

int check_device(const sdd_plan* p)
{
    int dev = -1;
    SDD_CUDA(cudaGetDevice(&dev));
    if (dev != p->device)
        return fail(SDD_ERR_INVALID_ARG, "plan belongs to another device than the current one");
    return SDD_OK;
}

int ensure_mc_buffers(sdd_plan* p, uint64_t items, cudaStream_t stream)
{
    AllocOn on(stream);
    if (!p->d_sums) {
        int rc;
        if ((rc = dev_alloc(&p->d_sums, (size_t)p->n_nodes))) return rc;
        if ((rc = dev_alloc(&p->d_mean, (size_t)p->n_nodes * 2))) return rc;
        if ((rc = dev_alloc(&p->d_stderr, (size_t)p->n_nodes * 2))) return rc;
        if ((rc = dev_alloc(&p->d_stats, 1))) return rc;
        if ((rc = dev_alloc(&p->d_queue, 1))) return rc;
    }
    if (items > p->slots_cap) {
        dev_free(p->d_slots, stream);
        p->slots_cap = 0;
        int rc = dev_alloc(&p->d_slots, (size_t)items);
        if (rc) return rc;
        p->slots_cap = items;
    }
    return SDD_OK;
}

// Solve buffers of a plan: allocation and the subdomain list only (no kernel),
// so that set-up never waits behind work running on the device.
int alloc_solve_buffers(sdd_plan* p, cudaStream_t stream)
{
    if (p->d_u) return SDD_OK;
    AllocOn on(stream);
    const int64_t nn = (int64_t)p->n * p->n;
    int rc;
    if ((rc = dev_alloc(&p->d_u, (size_t)nn * 2))) return rc;
    if ((rc = dev_alloc(&p->d_cx, (size_t)p->n * (p->n - 1)))) return rc;
    if ((rc = dev_alloc(&p->d_cy, (size_t)p->n * (p->n - 1)))) return rc;
    if ((rc = dev_alloc(&p->d_cxf, (size_t)p->n * (p->n - 1)))) return rc;
    if ((rc = dev_alloc(&p->d_cyf, (size_t)p->n * (p->n - 1)))) return rc;
    if ((rc = dev_alloc(&p->d_work, (size_t)nn * 11))) return rc;  // written before read
    if ((rc = dev_alloc(&p->d_mg, (size_t)std::max<int64_t>(p->mg_floats, 1)))) return rc;
    if ((rc = dev_alloc(&p->d_subs, p->h_subs.size()))) return rc;
    if ((rc = dev_alloc(&p->d_substats, p->h_subs.size()))) return rc;
    SDD_CUDA(cudaMemcpyAsync(p->d_subs, p->h_subs.data(), p->h_subs.size() * sizeof(SubDev),
                             cudaMemcpyHostToDevice, stream));
    return SDD_OK;
}

// Edge coefficients of a plan, computed once, on the stream of its first solve.
int ensure_coefs(sdd_plan* p, cudaStream_t stream)
{
    if (p->coefs_ready) return SDD_OK;
    int rc = launch_edge_coefs(p->n, p->dens.family, p->dens.coef_mode, p->dens.params,
                               p->d_tab64, p->dens.tn, p->d_cx,
                               p->d_cy, p->d_cxf, p->d_cyf, stream);
    if (rc) return rc;
    p->coefs_ready = true;
    return SDD_OK;
}

int ensure_solve_buffers(sdd_plan* p, cudaStream_t stream)
{
    int rc = alloc_solve_buffers(p, stream);
    if (rc) return rc;
    return ensure_coefs(p, stream);
}

// Paths per work item: enough items to spread over every warp slot of the
// device several times, at least 64 and at most 4096 paths per item.  It
// depends only on the mesh's own node count and N, so a mesh's sums are the
// same alone and inside a batch.
uint32_t auto_chunk(uint64_t paths, int64_t n_nodes)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    (void)dev;
    const double target = (double)paths * (double)n_nodes / (32.0 * 24.0 * (double)sms);
    uint32_t c = 64;
    while (c < 4096 && (double)(2 * c) <= target) c *= 2;
    const uint32_t cap = (uint32_t)(((paths + 31) / 32) * 32);
    return std::min(c, cap);
}

int validate_mc(const sdd_mc_params* mc)
{
    if (!mc) return fail(SDD_ERR_INVALID_ARG, "mc params are NULL");
    if (mc->paths_per_node < 2 || mc->paths_per_node >= (1ull << 32))
        return fail(SDD_ERR_INVALID_ARG, "paths_per_node must be in [2, 2^32)");
    if (!(mc->dt > 0.0) || !std::isfinite(mc->dt))
        return fail(SDD_ERR_INVALID_ARG, "dt must be positive and finite");
    if (mc->precision != SDD_FP64 && mc->precision != SDD_FP32_STEP)
        return fail(SDD_ERR_INVALID_ARG, "unknown precision");
    if (mc->chunk < 0 || mc->chunk > 8192 || (mc->chunk > 0 && mc->chunk % 32 != 0))
        return fail(SDD_ERR_INVALID_ARG, "chunk must be 0 or a multiple of 32 up to 8192");
    if (mc->exit_test != SDD_EXIT_END_OF_STEP && mc->exit_test != SDD_EXIT_BRIDGE)
        return fail(SDD_ERR_INVALID_ARG, "unknown exit_test");
    if (mc->stepper != SDD_STEP_EULER && mc->stepper != SDD_STEP_EXPONENTIAL)
        return fail(SDD_ERR_INVALID_ARG, "unknown stepper");
    const double cap = mc->max_steps ? (double)mc->max_steps : std::ceil(2.0 / mc->dt);
    if (cap < 1.0 || cap > 4294967294.0)
        return fail(SDD_ERR_INVALID_ARG, "max_steps must be in [1, 2^32 - 2]");
    if (mc->reserved != 0) return fail(SDD_ERR_INVALID_ARG, "reserved must be 0");
    if (mc->path_begin) {
        if (mc->path_begin > mc->paths_per_node)
            return fail(SDD_ERR_INVALID_ARG, "path_begin must not exceed paths_per_node");
        if (!mc->chunk || mc->path_begin % (uint64_t)mc->chunk)
            return fail(SDD_ERR_INVALID_ARG,
                        "a continued run needs an explicit chunk that divides path_begin");
    }
    return SDD_OK;
}

// A run with path_begin > 0 continues the plan's previous whole run: same
// request and parameters but N, which must equal path_begin.
int check_continuation(const sdd_plan* p, const sdd_mc_params* mc, int64_t nodes)
{
    if (!p->items_valid)
        return fail(SDD_ERR_INVALID_ARG,
                    "path_begin > 0 but the plan holds no previous whole run to continue");
    const sdd_mc_params& q = p->items_mc;
    auto cap = [](const sdd_mc_params& m) {
        return m.max_steps ? m.max_steps : (uint64_t)std::ceil(2.0 / m.dt);
    };
    auto tie = [](const sdd_mc_params& m) {
        return m.tie_delta >= 0.0 ? m.tie_delta : (m.precision == SDD_FP64 ? 1e-11 : 0.0);
    };
    if (q.paths_per_node != mc->path_begin)
        return fail(SDD_ERR_INVALID_ARG, "path_begin (" + std::to_string(mc->path_begin) +
                                             ") differs from the previous run's paths per node (" +
                                             std::to_string(q.paths_per_node) + ")");
    if (q.seed != mc->seed || q.dt != mc->dt || q.precision != mc->precision ||
        q.chunk != mc->chunk || cap(q) != cap(*mc) || tie(q) != tie(*mc) ||
        q.exit_test != mc->exit_test || q.stepper != mc->stepper || p->items_nodes != nodes)
        return fail(SDD_ERR_INVALID_ARG,
                    "path_begin > 0 but the previous run had other parameters than this one "
                    "(seed, dt, precision, chunk, step cap, tie delta, exit test, stepper)");
    return SDD_OK;
}

uint32_t chunk_of(const sdd_plan* p, const sdd_mc_params* mc)
{
    return mc->chunk ? (uint32_t)mc->chunk : auto_chunk(mc->paths_per_node, p->n_nodes);
}

// Mesh record of plan p for Monte Carlo parameters mc (outputs and offsets
// are set by the caller).
void mesh_record(const sdd_plan* p, const sdd_mc_params* mc, MeshDev& m)
{
    memset(&m, 0, sizeof(m));
    const uint32_t chunk = chunk_of(p, mc);
    m.n = p->n;
    m.family = p->dens.family;
    m.precision = mc->precision;
    m.key0 = (uint32_t)(mc->seed & 0xffffffffu);
    m.key1 = (uint32_t)(mc->seed >> 32);
    m.paths = (uint32_t)mc->paths_per_node;
    m.chunk = chunk;
    m.chunks_per_node = (uint32_t)((mc->paths_per_node + chunk - 1) / chunk);
    m.max_steps = (uint32_t)(mc->max_steps ? mc->max_steps : (uint64_t)std::ceil(2.0 / mc->dt));
    m.bridge = mc->exit_test == SDD_EXIT_BRIDGE ? 1 : 0;
    m.stepper = mc->stepper;
    m.n_nodes = p->n_nodes;
    m.dt = mc->dt;
    m.sqrt2dt = std::sqrt(2.0 * mc->dt);
    m.tie_delta = mc->tie_delta >= 0.0 ? mc->tie_delta : (mc->precision == SDD_FP64 ? 1e-11 : 0.0);
    m.nodes = p->d_nodes;
    m.edges = p->d_edges;
    fill_fp32_params(m, p->dens);
    m.tab64 = p->d_tab64;
    m.cell32 = p->d_cell32;
    m.tn = p->dens.tn;
    m.chunk_begin = mc->path_begin ? (uint32_t)(mc->path_begin / chunk) : 0u;
}

// Builds the mesh record and launches the path kernel + reduction.
// Launch record of plan p's Monte Carlo for mc (few-point aware), with the
// plan's buffers sized for it; `few` tells whether the interface is few-point.
int mc_args(sdd_plan* p, const sdd_mc_params* mc, double* mean_dev, double* stderr_dev,
            sdd_node_sums* sums_dev, McArgs& a, bool& few, cudaStream_t stream);

// Tail of a Monte Carlo run after the reduction: interpolation of a few-point
// interface, copies to the caller's device outputs, the plan's bookkeeping.
int mc_tail(sdd_plan* p, const sdd_mc_params* mc, bool few, double* mean_dev, double* stderr_dev,
            cudaStream_t stream)
{
    int rc;
    if (few) {
        if ((rc = launch_interp(p->d_interp, (int64_t)p->h_interp.size(), stream))) return rc;
        const size_t bytes = (size_t)p->n_nodes * 2 * sizeof(double);
        if (mean_dev && mean_dev != p->d_mean)
            SDD_CUDA(cudaMemcpyAsync(mean_dev, p->d_mean, bytes, cudaMemcpyDeviceToDevice, stream));
        if (stderr_dev && stderr_dev != p->d_stderr)
            SDD_CUDA(cudaMemcpyAsync(stderr_dev, p->d_stderr, bytes, cudaMemcpyDeviceToDevice, stream));
    }
    if (!p->mc_done) SDD_CUDA(cudaEventCreateWithFlags(&p->mc_done, cudaEventDisableTiming));
    SDD_CUDA(cudaEventRecord(p->mc_done, stream));
    p->last_paths = mc->paths_per_node;
    p->have_mc = true;
    p->last_stream = stream;
    return SDD_OK;
}

int run_mc(sdd_plan* p, const sdd_mc_params* mc, double* mean_dev, double* stderr_dev,
           sdd_node_sums* sums_dev, cudaStream_t stream)
{
    int rc = validate_mc(mc);
    if (rc) return rc;
    p->resume_active = false;                 // a whole run replaces any split one
    const int64_t nodes = p->n_mc;
    if (mc->path_begin) {
        // continue the previous run: its items move to their places in this
        // run's node-major layout (node v, chunk c at v * cpn + c)
        if ((rc = check_continuation(p, mc, nodes))) return rc;
        const uint32_t chunk = (uint32_t)mc->chunk;
        const uint64_t cpn_prev = mc->path_begin / chunk;
        const uint64_t cpn = (mc->paths_per_node + chunk - 1) / chunk;
        AllocOn on(stream);
        Slot* fresh = nullptr;
        if ((rc = dev_alloc(&fresh, (size_t)(nodes * cpn)))) return rc;
        if (nodes > 0)
            SDD_CUDA(cudaMemcpy2DAsync(fresh, cpn * sizeof(Slot), p->d_slots, cpn_prev * sizeof(Slot),
                                       cpn_prev * sizeof(Slot), (size_t)nodes,
                                       cudaMemcpyDeviceToDevice, stream));
        dev_free(p->d_slots, stream);
        p->d_slots = fresh;
        p->slots_cap = (uint64_t)nodes * cpn;
    }
    p->items_valid = false;
    McArgs a;
    bool few = false;
    if ((rc = mc_args(p, mc, mean_dev, stderr_dev, sums_dev, a, few, stream))) return rc;
    SDD_CUDA(cudaMemsetAsync(p->d_stats, 0, sizeof(McStatsDev), stream));
    if ((rc = launch_mc(a, mc->precision, mesh_kernel_class(a.single.family, a.single.nb,
                                                            a.single.stepper, mc->exit_test), stream)))
        return rc;
    p->items_valid = true;
    p->items_mc = *mc;
    p->items_nodes = nodes;
    ++p->items_run;
    return mc_tail(p, mc, few, mean_dev, stderr_dev, stream);
}

int mc_args(sdd_plan* p, const sdd_mc_params* mc, double* mean_dev, double* stderr_dev,
            sdd_node_sums* sums_dev, McArgs& a, bool& few, cudaStream_t stream)
{
    int rc;
    memset(&a, 0, sizeof(a));
    MeshDev& m = a.single;
    mesh_record(p, mc, m);
    few = p->n_mc < p->n_nodes;                      // few-point interface
    if (few) {
        m.n_nodes = p->n_mc;
        if (m.chunk == auto_chunk(mc->paths_per_node, p->n_nodes) && !mc->chunk) {
            m.chunk = auto_chunk(mc->paths_per_node, p->n_mc);
            m.chunks_per_node = (uint32_t)((mc->paths_per_node + m.chunk - 1) / m.chunk);
        }
    }
    const uint64_t items = (uint64_t)m.n_nodes * m.chunks_per_node;
    if ((rc = ensure_mc_buffers(p, items, stream))) return rc;
    m.nodes = few ? p->d_mc_nodes : p->d_nodes;
    m.node_ids = few ? p->d_mc_ids : nullptr;
    m.edges = p->d_edges;
    m.sums = sums_dev ? sums_dev : p->d_sums;
    // interpolation reads the plan's own output buffers
    m.mean = few ? p->d_mean : (mean_dev ? mean_dev : p->d_mean);
    m.stderr_ = few ? p->d_stderr : (stderr_dev ? stderr_dev : p->d_stderr);
    m.stats = p->d_stats;
    if (few && m.sums)
        SDD_CUDA(cudaMemsetAsync(m.sums, 0, (size_t)p->n_nodes * sizeof(sdd_node_sums), stream));
    for (int r = 0; r < 10; ++r) {
        a.rk[2 * r] = m.key0 + (uint32_t)r * 0x9E3779B9u;
        a.rk[2 * r + 1] = m.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    a.meshes = nullptr;
    a.n_meshes = 1;
    a.total_items = items;
    a.total_nodes = (uint64_t)m.n_nodes;
    a.queue = p->d_queue;
    a.slots = p->d_slots;
    return SDD_OK;
}

int stats_from_dev(const McStatsDev& s, uint64_t paths, sdd_mc_stats* out)
{
    out->paths = paths;
    out->path_steps = s.steps;
    out->ties = s.ties;
    out->non_exits = s.caps;
    double se;
    memcpy(&se, &s.max_stderr_bits, sizeof(se));
    out->max_stderr = se;
    if (s.lost != 0)
        return fail(SDD_ERR_CUDA, "internal error: a node's path count differs from N");
    return SDD_OK;
}

int read_mc_stats(sdd_plan* p, sdd_mc_stats* out, cudaStream_t stream)
{
    McStatsDev s;
    SDD_CUDA(cudaMemcpyAsync(&s, p->d_stats, sizeof(s), cudaMemcpyDeviceToHost, stream));
    SDD_CUDA(cudaStreamSynchronize(stream));
    return stats_from_dev(s, p->last_paths * (uint64_t)p->n_mc, out);
}

// Bit of a solver in a launch's solver mask (1 SOR, 2 multigrid CG, 4 Jacobi CG).
int solver_bit(int solver)
{
    return solver == SDD_SOLVER_SOR ? 1 : solver == SDD_SOLVER_CG_FP32_REFINE ? 2 : 4;
}

int validate_solve(const sdd_solve_params* sp)
{
    if (!sp) return fail(SDD_ERR_INVALID_ARG, "solve params are NULL");
    if (sp->solver != SDD_SOLVER_SOR && sp->solver != SDD_SOLVER_CG_FP32_REFINE &&
        sp->solver != SDD_SOLVER_CG_JACOBI_FP32_REFINE)
        return fail(SDD_ERR_INVALID_ARG, "unknown solver");
    if (!(sp->tol > 0.0) || !std::isfinite(sp->tol))
        return fail(SDD_ERR_INVALID_ARG, "tol must be positive");
    if (sp->max_iter < 0) return fail(SDD_ERR_INVALID_ARG, "max_iter must be >= 0");
    if (!(sp->omega == 0.0 || (sp->omega > 0.0 && sp->omega < 2.0)))
        return fail(SDD_ERR_INVALID_ARG, "omega must be 0 or in (0, 2)");
    if (sp->block_threads != 0 && sp->block_threads != 256 && sp->block_threads != 512 &&
        sp->block_threads != 1024)
        return fail(SDD_ERR_INVALID_ARG, "block_threads must be 0, 256, 512 or 1024");
    return SDD_OK;
}

// Fills the mesh from the boundary tables and device interface values, then
// solves every subdomain.  Result in p->d_u.
int run_solve(sdd_plan* p, const double* iface_dev, const sdd_solve_params* sp,
              cudaStream_t stream)
{
    int rc = validate_solve(sp);
    if (rc) return rc;
    if ((rc = ensure_solve_buffers(p, stream))) return rc;
    SolveMeshDev sm;
    memset(&sm, 0, sizeof(sm));
    sm.n = p->n;
    sm.solver = sp->solver;
    sm.max_iter = sp->max_iter > 0 ? sp->max_iter : (sp->solver == SDD_SOLVER_SOR ? 200000 : 20000);
    sm.tol = sp->tol;
    sm.omega = sp->omega;
    sm.u = p->d_u;
    sm.cx = p->d_cx;
    sm.cy = p->d_cy;
    sm.cxf = p->d_cxf;
    sm.cyf = p->d_cyf;
    sm.work = p->d_work;
    sm.mg = p->d_mg;
    if ((rc = launch_fill_mesh(p->n, p->d_edges, p->d_nodes, p->n_nodes, iface_dev, p->d_u,
                               p->d_subs, (int)p->h_subs.size(), stream)))
        return rc;
    SolveArgs a;
    a.meshes = nullptr;
    a.single = sm;
    a.subs = p->d_subs;
    a.n_subs = (int)p->h_subs.size();
    a.solver_mask = solver_bit(sp->solver);
    a.threads = sp->block_threads;
    a.stats = p->d_substats;
    if ((rc = launch_solve(a, stream))) return rc;
    p->last_stream = stream;
    return SDD_OK;
}

int read_solve_stats(sdd_plan* p, sdd_solve_stats* out, cudaStream_t stream)
{
    std::vector<SubStat> st(p->h_subs.size());
    if (!st.empty())
        SDD_CUDA(cudaMemcpyAsync(st.data(), p->d_substats, st.size() * sizeof(SubStat),
                                 cudaMemcpyDeviceToHost, stream));
    SDD_CUDA(cudaStreamSynchronize(stream));
    out->subdomains = (int32_t)st.size();
    out->converged = 0;
    out->max_iterations = 0;
    out->max_rel_residual = 0.0;
    out->node_iterations = 0.0;
    for (const SubStat& s : st) {
        out->converged += s.converged;
        out->max_iterations = std::max(out->max_iterations, s.iterations);
        out->max_rel_residual = std::max(out->max_rel_residual, s.rel_residual);
    }
    for (const SubDev& d : p->h_subs)
        out->node_iterations += (double)st[d.slot].iterations * interior_nodes(d);
    return out->converged == out->subdomains
               ? SDD_OK
               : fail(SDD_ERR_NOT_CONVERGED, "a subdomain did not reach the tolerance");
}

// ----------------------------------------------------- few-point interface --
// Monte Carlo nodes of a placement (§3.6): every crossing of two interface
// lines, plus per line either k equispaced points (positions
// round(r (m-1)/(k+1)), r = 1..k, m = points on the line including its two
// boundary ends) or the nodes where the first or the second centred
// difference of the density w along the line has a local extremum.
std::vector<uint8_t> placement_mask(const sdd_plan* p, int mode, int k)
{
    const int n = p->n;
    std::vector<uint8_t> mask(p->n_nodes, mode == SDD_PLACE_ALL ? 1 : 0);
    if (mode == SDD_PLACE_ALL) return mask;
    std::vector<int64_t> index((size_t)n * n, -1);
    for (int64_t q = 0; q < p->n_nodes; ++q)
        index[(size_t)p->h_nodes[2 * q + 1] * n + p->h_nodes[2 * q]] = q;
    std::vector<char> onx(n, 0), ony(n, 0);
    for (int v : p->ix) onx[v] = 1;
    for (int v : p->iy) ony[v] = 1;
    for (int64_t q = 0; q < p->n_nodes; ++q)
        if (onx[p->h_nodes[2 * q]] && ony[p->h_nodes[2 * q + 1]]) mask[q] = 1;
    sdd_density w = p->dens;
    w.coef_mode = SDD_COEF_W;
    const double h = 1.0 / (double)(n - 1);
    auto mark_line = [&](bool vertical, int line) {
        const int m = n;
        auto node_at = [&](int r) -> int64_t {
            return vertical ? index[(size_t)r * n + line] : index[(size_t)line * n + r];
        };
        std::vector<int> chosen;
        if (mode == SDD_PLACE_EQUISPACED) {
            for (int r = 1; r <= k; ++r) chosen.push_back((int)((2LL * r * (m - 1) + (k + 1)) / (2LL * (k + 1))));
        } else {
            std::vector<double> rho(m), d1(m, 0.0), d2(m, 0.0);
            for (int r = 0; r < m; ++r) {
                const double a = (double)line * h, b = (double)r * h;
                rho[r] = vertical ? host_coef(w, a, b) : host_coef(w, b, a);
            }
            for (int r = 1; r < m - 1; ++r) {
                d1[r] = (rho[r + 1] - rho[r - 1]) / (2 * h);
                d2[r] = (rho[r + 1] - 2 * rho[r] + rho[r - 1]) / (h * h);
            }
            for (const std::vector<double>* dv : {&d1, &d2}) {
                const std::vector<double>& d = *dv;
                for (int r = 2; r < m - 2; ++r)
                    if ((d[r] > d[r - 1] && d[r] >= d[r + 1]) || (d[r] < d[r - 1] && d[r] <= d[r + 1]))
                        chosen.push_back(r);
            }
        }
        for (int r : chosen)
            if (r >= 1 && r <= m - 2) {
                const int64_t q = node_at(r);
                if (q >= 0) mask[q] = 1;
            }
    };
    for (int v : p->ix) mark_line(true, v);
    for (int v : p->iy) mark_line(false, v);
    return mask;
}

// Interpolation entries of the non-Monte-Carlo interface nodes: along each
// line, between the nearest Monte Carlo nodes (or the line's boundary ends,
// boundary map); vertical lines first.
std::vector<InterpEntry> interp_entries(const sdd_plan* p, const std::vector<uint8_t>& mask)
{
    const int n = p->n;
    std::vector<int64_t> index((size_t)n * n, -1);
    for (int64_t q = 0; q < p->n_nodes; ++q)
        index[(size_t)p->h_nodes[2 * q + 1] * n + p->h_nodes[2 * q]] = q;
    auto bvalue = [&](int i, int j, int c) -> double {
        // boundary grid: rows j = 0, n-1 from the bottom/top tables, else columns
        const auto E = [&](int comp, int edge, int kk) { return p->h_edges[((size_t)comp * 4 + edge) * n + kk]; };
        if (j == 0) return E(c, 0, i);
        if (j == n - 1) return E(c, 1, i);
        if (i == 0) return E(c, 2, j);
        return E(c, 3, j);
    };
    std::vector<InterpEntry> out;
    auto do_line = [&](bool vertical, int line) {
        auto ij = [&](int r, int& i, int& j) { if (vertical) { i = line; j = r; } else { i = r; j = line; } };
        std::vector<int> known;
        for (int r = 0; r < n; ++r) {
            int i, j;
            ij(r, i, j);
            if (r == 0 || r == n - 1) { known.push_back(r); continue; }
            const int64_t q = index[(size_t)j * n + i];
            if (q >= 0 && mask[q]) known.push_back(r);
        }
        for (size_t kk = 0; kk + 1 < known.size(); ++kk) {
            const int ra = known[kk], rb = known[kk + 1];
            for (int r = ra + 1; r < rb; ++r) {
                int i, j, ia, ja, ib, jb;
                ij(r, i, j);
                ij(ra, ia, ja);
                ij(rb, ib, jb);
                InterpEntry e;
                memset(&e, 0, sizeof(e));
                e.q = index[(size_t)j * n + i];
                e.w = (double)(r - ra) / (double)(rb - ra);
                e.a = (ra == 0 || ra == n - 1) ? -1 : index[(size_t)ja * n + ia];
                e.b = (rb == 0 || rb == n - 1) ? -1 : index[(size_t)jb * n + ib];
                for (int c = 0; c < 2; ++c) {
                    e.ca[c] = e.a < 0 ? bvalue(ia, ja, c) : 0.0;
                    e.cb[c] = e.b < 0 ? bvalue(ib, jb, c) : 0.0;
                }
                out.push_back(e);
            }
        }
    };
    for (int v : p->ix) do_line(true, v);
    for (int v : p->iy) do_line(false, v);
    return out;
}

// ------------------------------------------------------------------ batch --
// Many plans generated together: one path-kernel launch per (precision,
// density class) group over all their interface nodes, one reduction per
// group, one Dirichlet-fill launch and one solve launch over every subdomain
// of every mesh.  Everything a run needs lives on the device from creation
// on, so a run is a fixed sequence of memsets and kernel launches, which can
// be captured once into a CUDA graph and replayed.
struct McGroup {
    int precision;
    int kc;                 // kernel class (density class + KC_EXPO)
    int blocks;                 // persistent grid
    McArgs args;
};

// A plan whose run continues its previous single-plan run (path_begin > 0):
// before the path kernels, the previous run's items (rows of cpn_prev slots
// in the plan's buffer) are copied to their places in the batch's slots
// (rows of cpn), where the path kernel skips them.
struct SlotSeed {
    const sdd_plan* plan;
    uint64_t run;           // the plan's run whose items are copied (items_run)
    const Slot* src;
    uint64_t dst;           // first slot of the plan's mesh in the batch's slots
    uint64_t cpn_prev, cpn, rows;
};

}  // namespace
}  // namespace sdd

struct sdd_batch {
    int device = 0;
    std::vector<sdd_plan*> plans;
    std::vector<uint64_t> plan_paths;           // N per plan
    std::vector<sdd::McGroup> groups;
    std::vector<sdd::SlotSeed> seeds;           // plans that continue a previous run
    std::vector<int> plan_slot;                 // plan -> index of its record in d_meshes
    sdd::MeshDev* d_meshes = nullptr;
    uint64_t* d_offs = nullptr;                 // item and node prefix sums of every group
    sdd::Slot* d_slots = nullptr;
    unsigned long long* d_queues = nullptr;     // one work counter per group
    sdd::McStatsDev* d_stats = nullptr;         // one per plan
    sdd::FillDev* d_fill = nullptr;
    uint64_t* d_fill_off = nullptr;
    uint64_t fill_total = 0;
    sdd::SolveMeshDev* d_smesh = nullptr;
    sdd::SubDev* d_subs = nullptr;
    sdd::SubStat* d_substats = nullptr;
    sdd::InterpEntry* d_interp = nullptr;       // few-point interfaces of the plans
    int64_t n_interp = 0;
    std::vector<int> sub_begin;                 // plan -> first subdomain
    int n_subs = 0;
    int solver_mask = 0;                        // solvers used by the batch's plans
    int solve_threads = 0;                      // largest CTA size requested (0: default)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    uint64_t graph_kernels = 0;                 // kernels in one replay of the graph
    cudaStream_t last_stream = nullptr;
    bool ran = false;
};

namespace sdd {
namespace {

void batch_free(sdd_batch* b)
{
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    const cudaStream_t fs = b->ran ? b->last_stream : setup_stream();
    dev_free(b->d_meshes, fs);
    dev_free(b->d_offs, fs);
    dev_free(b->d_slots, fs);
    dev_free(b->d_queues, fs);
    dev_free(b->d_stats, fs);
    dev_free(b->d_fill, fs);
    dev_free(b->d_fill_off, fs);
    dev_free(b->d_smesh, fs);
    dev_free(b->d_subs, fs);
    dev_free(b->d_substats, fs);
    dev_free(b->d_interp, fs);
    delete b;
}

// The plans that continue a previous run must still hold that run's items
// where the batch was told they are.
int check_seeds(const sdd_batch* b)
{
    for (const SlotSeed& q : b->seeds)
        if (!q.plan->items_valid || q.plan->items_run != q.run || q.plan->d_slots != q.src)
            return fail(SDD_ERR_INVALID_ARG,
                        "a plan of the batch continues a run (path_begin > 0) whose work items "
                        "it no longer holds (another Monte Carlo ran on it since)");
    return SDD_OK;
}

// Enqueues one whole run of the batch on `stream` (no host synchronisation,
// no device queries: safe inside a stream capture).
int batch_enqueue(sdd_batch* b, cudaStream_t stream, int phases = 3)
{
    const size_t np = b->plans.size();
    if (phases & 1) {
        SDD_CUDA(cudaMemsetAsync(b->d_stats, 0, np * sizeof(McStatsDev), stream));
        for (const SlotSeed& q : b->seeds)
            if (q.rows)
                SDD_CUDA(cudaMemcpy2DAsync(b->d_slots + q.dst, q.cpn * sizeof(Slot), q.src,
                                           q.cpn_prev * sizeof(Slot), q.cpn_prev * sizeof(Slot),
                                           (size_t)q.rows, cudaMemcpyDeviceToDevice, stream));
        for (const McGroup& g : b->groups) {
            int rc = launch_mc_sized(g.args, g.precision, g.kc, g.blocks, stream);
            if (rc) return rc;
        }
        int rc = launch_interp(b->d_interp, b->n_interp, stream);
        if (rc) return rc;
    }
    if (phases & 2) {
        for (sdd_plan* p : b->plans) {                 // first solve: edge coefficients
            int rc = ensure_coefs(p, stream);
            if (rc) return rc;
        }
        int rc = launch_fill_batched(b->d_fill, b->d_fill_off, (int)np, b->fill_total, stream);
        if (rc) return rc;
        SolveArgs sa;
        memset(&sa, 0, sizeof(sa));
        sa.meshes = b->d_smesh;
        sa.subs = b->d_subs;
        sa.n_subs = b->n_subs;
        sa.solver_mask = b->solver_mask;
        sa.threads = b->solve_threads;
        sa.stats = b->d_substats;
        return launch_solve(sa, stream);
    }
    return SDD_OK;
}

}  // namespace
}  // namespace sdd

using namespace sdd;

extern "C" {

int sdd_mesh_plan(int n, int sx, int sy, const sdd_density* dens, const sdd_bmap* bmap,
                  sdd_plan** out)
{
    NvtxRange nvtx_range("sdd_mesh_plan");
    clear_error();
    if (!out) return fail(SDD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 3 || n > 16385) return fail(SDD_ERR_INVALID_ARG, "n must be in [3, 16385]");
    if (sx < 1 || sy < 1 || sx > n - 1 || sy > n - 1)
        return fail(SDD_ERR_INVALID_ARG, "sx, sy must be in [1, n-1]");
    int rc = validate_density(dens);
    if (rc) return rc;
    if (!bmap) return fail(SDD_ERR_INVALID_ARG, "bmap is NULL");
    if (bmap->mode != SDD_BMAP_IDENTITY && bmap->mode != SDD_BMAP_PAPER_1D &&
        bmap->mode != SDD_BMAP_TABLE)
        return fail(SDD_ERR_INVALID_ARG, "unknown boundary-map mode");
    if (bmap->mode == SDD_BMAP_TABLE && !bmap->edges)
        return fail(SDD_ERR_INVALID_ARG, "TABLE boundary map needs edges");

    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(SDD_ERR_NO_DEVICE, "no CUDA device");
    }
    sdd_plan* p = new (std::nothrow) sdd_plan();
    if (!p) return fail(SDD_ERR_OOM, "host allocation failed");
    cudaGetDevice(&p->device);
    p->n = n;
    p->sx = sx;
    p->sy = sy;
    p->dens = *dens;
    for (int q = dens->n_params; q < SDD_MAX_PARAMS; ++q) p->dens.params[q] = 0.0;
    if (dens->family == SDD_FAMILY_TABLE) {               // the plan keeps its own copy
        p->h_table.assign(dens->table, dens->table + (size_t)dens->tn * dens->tn);
        p->dens.table = p->h_table.data();
    } else {
        p->dens.table = nullptr;
        p->dens.tn = 0;
    }
    p->bmap_mode = bmap->mode;
    p->ix = interface_lines(n, sx);
    p->iy = interface_lines(n, sy);

    // interface nodes, ordered by j then i
    std::vector<char> onx(n, 0), ony(n, 0);
    for (int v : p->ix) onx[v] = 1;
    for (int v : p->iy) ony[v] = 1;
    for (int j = 1; j < n - 1; ++j)
        for (int i = 1; i < n - 1; ++i)
            if (onx[i] || ony[j]) {
                p->h_nodes.push_back(i);
                p->h_nodes.push_back(j);
            }
    p->n_nodes = (int64_t)p->h_nodes.size() / 2;
    p->n_mc = p->n_nodes;
    p->h_mask.assign(p->n_nodes, 1);

    // subdomain boxes
    std::vector<int> X{0}, Y{0};
    X.insert(X.end(), p->ix.begin(), p->ix.end());
    X.push_back(n - 1);
    Y.insert(Y.end(), p->iy.begin(), p->iy.end());
    Y.push_back(n - 1);
    for (int b = 0; b < sy; ++b)
        for (int a = 0; a < sx; ++a) {
            const int32_t slot = (int32_t)p->h_subs.size();
            MgShape mg;
            mg_shape(X[a + 1] - X[a] - 1, Y[b + 1] - Y[b] - 1, mg);
            p->h_subs.push_back(SubDev{0, X[a], X[a + 1], Y[b], Y[b + 1], slot, p->mg_floats});
            p->mg_floats += mg.total;
        }
    sort_largest_first(p->h_subs);

    // boundary tables [2][4][n]
    p->h_edges.assign((size_t)8 * n, 0.0);
    auto E = [&](int c, int edge, int k) -> double& { return p->h_edges[((size_t)c * 4 + edge) * n + k]; };
    if (bmap->mode == SDD_BMAP_TABLE) {
        for (size_t q = 0; q < p->h_edges.size(); ++q) {
            if (!std::isfinite(bmap->edges[q])) {
                delete p;
                return fail(SDD_ERR_INVALID_ARG, "non-finite boundary table value");
            }
            p->h_edges[q] = bmap->edges[q];
        }
    } else {
        for (int k = 0; k < n; ++k) {
            const double x = (double)k / (double)(n - 1);
            E(0, 0, k) = x; E(0, 1, k) = x; E(0, 2, k) = 0.0; E(0, 3, k) = 1.0;
            E(1, 0, k) = 0.0; E(1, 1, k) = 1.0; E(1, 2, k) = x; E(1, 3, k) = x;
        }
        if (bmap->mode == SDD_BMAP_PAPER_1D) {
            // u_k = sum_{m<k} 1/c_{m+1/2} / sum_m 1/c_{m+1/2} along each edge
            for (int edge = 0; edge < 4; ++edge) {
                const int comp = edge < 2 ? 0 : 1;
                std::vector<double> cum(n, 0.0);
                for (int m = 0; m < n - 1; ++m) {
                    const double mid = ((double)m + 0.5) / (double)(n - 1);
                    double s, t;
                    if (edge == 0) { s = mid; t = 0.0; }
                    else if (edge == 1) { s = mid; t = 1.0; }
                    else if (edge == 2) { s = 0.0; t = mid; }
                    else { s = 1.0; t = mid; }
                    cum[m + 1] = cum[m] + 1.0 / host_coef(p->dens, s, t);
                }
                for (int k = 0; k < n; ++k) E(comp, edge, k) = cum[k] / cum[n - 1];
            }
        }
    }

    const cudaStream_t ss = setup_stream();
    {
        AllocOn on(ss);
        if ((rc = dev_alloc(&p->d_nodes, (size_t)std::max<int64_t>(p->n_nodes, 1))) ||
            (rc = dev_alloc(&p->d_edges, p->h_edges.size())) ||
            (!p->h_table.empty() &&
             ((rc = dev_alloc(&p->d_tab64, p->h_table.size())) ||
              (rc = dev_alloc(&p->d_cell32, (size_t)(p->dens.tn - 1) * (p->dens.tn - 1)))))) {
            sdd_plan_destroy(p);
            return rc;
        }
    }
    // FP32 stepping reads one 16-byte record per cell: the bilinear
    // interpolant's gradient coefficients, scaled by 1/spacing (FP64, rounded)
    std::vector<float4> cells;
    if (!p->h_table.empty()) {
        const int tn = p->dens.tn;
        const double m = (double)(tn - 1);
        const double* T = p->h_table.data();
        cells.resize((size_t)(tn - 1) * (tn - 1));
        for (int b = 0; b < tn - 1; ++b)
            for (int a = 0; a < tn - 1; ++a) {
                const double L00 = T[b * tn + a], L10 = T[b * tn + a + 1];
                const double L01 = T[(b + 1) * tn + a], L11 = T[(b + 1) * tn + a + 1];
                cells[(size_t)b * (tn - 1) + a] =
                    make_float4((float)((L10 - L00) * m), (float)((L01 - L00) * m),
                                (float)((L11 - L10 - L01 + L00) * m), 0.0f);
            }
    }
    cudaError_t ce = cudaSuccess;
    if (!p->h_table.empty()) {
        ce = cudaMemcpyAsync(p->d_tab64, p->h_table.data(), p->h_table.size() * sizeof(double),
                             cudaMemcpyHostToDevice, ss);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(p->d_cell32, cells.data(), cells.size() * sizeof(float4),
                                 cudaMemcpyHostToDevice, ss);
    }
    if (ce == cudaSuccess && p->n_nodes > 0)
        ce = cudaMemcpyAsync(p->d_nodes, p->h_nodes.data(), p->h_nodes.size() * sizeof(int32_t),
                             cudaMemcpyHostToDevice, ss);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(p->d_edges, p->h_edges.data(), p->h_edges.size() * sizeof(double),
                             cudaMemcpyHostToDevice, ss);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(ss);
    if (ce != cudaSuccess) {
        rc = cuda_status(ce, "cudaMemcpy(plan tables)");
        sdd_plan_destroy(p);
        return rc;
    }
    *out = p;
    return SDD_OK;
}

int sdd_plan_num_nodes(const sdd_plan* plan, int64_t* n_nodes)
{
    clear_error();
    if (!plan || !n_nodes) return fail(SDD_ERR_INVALID_ARG, "NULL argument");
    *n_nodes = plan->n_nodes;
    return SDD_OK;
}

int sdd_plan_nodes(const sdd_plan* plan, int32_t* ij)
{
    clear_error();
    if (!plan || !ij) return fail(SDD_ERR_INVALID_ARG, "NULL argument");
    std::copy(plan->h_nodes.begin(), plan->h_nodes.end(), ij);
    return SDD_OK;
}

int sdd_plan_edges(const sdd_plan* plan, double* edges)
{
    clear_error();
    if (!plan || !edges) return fail(SDD_ERR_INVALID_ARG, "NULL argument");
    std::copy(plan->h_edges.begin(), plan->h_edges.end(), edges);
    return SDD_OK;
}

int sdd_interface_mc(sdd_plan* p, const sdd_mc_params* mc, double* mean, double* stderr_,
                     sdd_mc_stats* stats, void* stream_)
{
    NvtxRange nvtx_range("sdd_interface_mc");
    clear_error();
    if (!p) return fail(SDD_ERR_INVALID_ARG, "plan is NULL");
    int rc = check_device(p);
    if (rc) return rc;
    cudaStream_t stream = as_stream(stream_);
    const bool mean_dev = is_device_ptr(mean), se_dev = is_device_ptr(stderr_);
    if ((rc = run_mc(p, mc, mean_dev ? mean : nullptr, se_dev ? stderr_ : nullptr, nullptr, stream)))
        return rc;
    const size_t bytes = (size_t)p->n_nodes * 2 * sizeof(double);
    bool host = false;
    if (mean && !mean_dev && bytes) {
        SDD_CUDA(cudaMemcpyAsync(mean, p->d_mean, bytes, cudaMemcpyDeviceToHost, stream));
        host = true;
    }
    if (stderr_ && !se_dev && bytes) {
        SDD_CUDA(cudaMemcpyAsync(stderr_, p->d_stderr, bytes, cudaMemcpyDeviceToHost, stream));
        host = true;
    }
    if (stats) return read_mc_stats(p, stats, stream);
    if (host) SDD_CUDA(cudaStreamSynchronize(stream));
    return SDD_OK;
}

int sdd_interface_mc_sums(sdd_plan* p, const sdd_mc_params* mc, sdd_node_sums* sums,
                          void* stream_)
{
    NvtxRange nvtx_range("sdd_interface_mc_sums");
    clear_error();
    if (!p || !sums) return fail(SDD_ERR_INVALID_ARG, "NULL argument");
    int rc = check_device(p);
    if (rc) return rc;
    cudaStream_t stream = as_stream(stream_);
    const bool dev = is_device_ptr(sums);
    if ((rc = run_mc(p, mc, nullptr, nullptr, dev ? sums : nullptr, stream))) return rc;
    if (!dev && p->n_nodes > 0) {
        SDD_CUDA(cudaMemcpyAsync(sums, p->d_sums, (size_t)p->n_nodes * sizeof(sdd_node_sums),
                                 cudaMemcpyDeviceToHost, stream));
        SDD_CUDA(cudaStreamSynchronize(stream));
    }
    return SDD_OK;
}

// ---- a Monte Carlo run split over calls, and its checkpoints ----
namespace {
constexpr uint32_t kCheckpointMagic = 0x43444453u;   // "SDDC"

struct CheckpointHeader {
    uint32_t magic, version;
    uint64_t n, n_mc, items_total, items_done, slot_bytes, plan_hash;
    sdd_mc_params mc;
};

// FNV-1a over what fixes a plan's Monte Carlo: grid, density, boundary tables,
// Monte Carlo nodes.
uint64_t plan_hash(const sdd_plan* p)
{
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void* data, size_t bytes) {
        const unsigned char* c = static_cast<const unsigned char*>(data);
        for (size_t q = 0; q < bytes; ++q) h = (h ^ c[q]) * 1099511628211ull;
    };
    mix(&p->n, sizeof(p->n));
    mix(&p->sx, sizeof(p->sx));
    mix(&p->sy, sizeof(p->sy));
    mix(&p->dens.family, sizeof(p->dens.family));
    mix(&p->dens.coef_mode, sizeof(p->dens.coef_mode));
    mix(p->dens.params, sizeof(p->dens.params));
    mix(p->h_table.data(), p->h_table.size() * sizeof(double));
    mix(p->h_edges.data(), p->h_edges.size() * sizeof(double));
    mix(p->h_mask.data(), p->h_mask.size());
    return h;
}

bool same_mc(const sdd_mc_params& a, const sdd_mc_params& b)
{
    return memcmp(&a, &b, sizeof(sdd_mc_params)) == 0;
}
}  // namespace

int sdd_interface_mc_advance(sdd_plan* p, const sdd_mc_params* mc, uint64_t max_items,
                             uint64_t* items_done, uint64_t* items_total, void* stream_)
{
    NvtxRange nvtx_range("sdd_interface_mc_advance");
    clear_error();
    if (!p || !mc) return fail(SDD_ERR_INVALID_ARG, "NULL argument");
    int rc = check_device(p);
    if (rc) return rc;
    if ((rc = validate_mc(mc))) return rc;
    if (mc->path_begin)
        return fail(SDD_ERR_INVALID_ARG, "a split run starts at path 0 (path_begin must be 0)");
    cudaStream_t stream = as_stream(stream_);
    McArgs a;
    bool few = false;
    p->items_valid = false;                      // the split run writes the item slots
    if ((rc = mc_args(p, mc, nullptr, nullptr, nullptr, a, few, stream))) return rc;
    if (!p->resume_active || !same_mc(p->resume_mc, *mc)) {     // a new split run
        p->resume_active = true;
        p->resume_mc = *mc;
        p->resume_next = 0;
        p->resume_total = a.total_items;
    }
    const uint64_t end = std::min(p->resume_total, p->resume_next + max_items);
    a.item_base = p->resume_next;
    a.total_items = end;
    if ((rc = launch_mc_paths(a, mc->precision,
                              mesh_kernel_class(a.single.family, a.single.nb, a.single.stepper,
                                                mc->exit_test),
                              stream)))
        return rc;
    p->resume_next = end;
    p->last_stream = stream;
    if (items_done) *items_done = p->resume_next;
    if (items_total) *items_total = p->resume_total;
    return SDD_OK;
}

int sdd_interface_mc_finish(sdd_plan* p, const sdd_mc_params* mc, double* mean, double* stderr_,
                            sdd_mc_stats* stats, void* stream_)
{
    NvtxRange nvtx_range("sdd_interface_mc_finish");
    clear_error();
    if (!p || !mc) return fail(SDD_ERR_INVALID_ARG, "NULL argument");
    int rc = check_device(p);
    if (rc) return rc;
    if (!p->resume_active || !same_mc(p->resume_mc, *mc))
        return fail(SDD_ERR_INVALID_ARG, "no split Monte Carlo run with these parameters");
    if (p->resume_next != p->resume_total)
        return fail(SDD_ERR_INVALID_ARG, "the split run has work items left: " +
                                             std::to_string(p->resume_total - p->resume_next));
    cudaStream_t stream = as_stream(stream_);
    const bool mean_dev = is_device_ptr(mean), se_dev = is_device_ptr(stderr_);
    McArgs a;
    bool few = false;
    if ((rc = mc_args(p, mc, mean_dev ? mean : nullptr, se_dev ? stderr_ : nullptr, nullptr, a,
                      few, stream)))
        return rc;
    SDD_CUDA(cudaMemsetAsync(p->d_stats, 0, sizeof(McStatsDev), stream));
    if ((rc = launch_mc_reduce(a, stream))) return rc;
    if ((rc = mc_tail(p, mc, few, mean_dev ? mean : nullptr, se_dev ? stderr_ : nullptr, stream)))
        return rc;
    p->resume_active = false;
    const size_t bytes = (size_t)p->n_nodes * 2 * sizeof(double);
    bool host = false;
    if (mean && !mean_dev && bytes) {
        SDD_CUDA(cudaMemcpyAsync(mean, p->d_mean, bytes, cudaMemcpyDeviceToHost, stream));
        host = true;
    }
    if (stderr_ && !se_dev && bytes) {
        SDD_CUDA(cudaMemcpyAsync(stderr_, p->d_stderr, bytes, cudaMemcpyDeviceToHost, stream));
        host = true;
    }
    if (stats) return read_mc_stats(p, stats, stream);
    if (host) SDD_CUDA(cudaStreamSynchronize(stream));
    return SDD_OK;
}

int sdd_mc_checkpoint_bytes(const sdd_plan* p, uint64_t* bytes)
{
    clear_error();
    if (!p || !bytes) return fail(SDD_ERR_INVALID_ARG, "NULL argument");
    if (!p->resume_active) return fail(SDD_ERR_INVALID_ARG, "no split Monte Carlo run to save");
    *bytes = sizeof(CheckpointHeader) + p->resume_next * sizeof(Slot);
    return SDD_OK;
}

int sdd_mc_checkpoint_save(sdd_plan* p, void* host, uint64_t bytes, void* stream_)
{
    NvtxRange nvtx_range("sdd_mc_checkpoint_save");
    clear_error();
    if (!p || !host) return fail(SDD_ERR_INVALID_ARG, "NULL argument");
    if (!p->resume_active) return fail(SDD_ERR_INVALID_ARG, "no split Monte Carlo run to save");
    const uint64_t need = sizeof(CheckpointHeader) + p->resume_next * sizeof(Slot);
    if (bytes < need)
        return fail(SDD_ERR_INVALID_ARG, "checkpoint buffer too small: " + std::to_string(need) +
                                             " bytes needed");
    int rc = check_device(p);
    if (rc) return rc;
    cudaStream_t stream = as_stream(stream_);
    CheckpointHeader h;
    memset(&h, 0, sizeof(h));
    h.magic = kCheckpointMagic;
    h.version = 2;
    h.n = (uint64_t)p->n;
    h.n_mc = (uint64_t)p->n_mc;
    h.items_total = p->resume_total;
    h.items_done = p->resume_next;
    h.slot_bytes = sizeof(Slot);
    h.plan_hash = plan_hash(p);
    h.mc = p->resume_mc;
    memcpy(host, &h, sizeof(h));
    if (p->resume_next)
        SDD_CUDA(cudaMemcpyAsync(static_cast<unsigned char*>(host) + sizeof(h), p->d_slots,
                                 p->resume_next * sizeof(Slot), cudaMemcpyDeviceToHost, stream));
    SDD_CUDA(cudaStreamSynchronize(stream));
    return SDD_OK;
}

int sdd_mc_checkpoint_load(sdd_plan* p, const void* host, uint64_t bytes, void* stream_)
{
    NvtxRange nvtx_range("sdd_mc_checkpoint_load");
    clear_error();
    if (!p || !host) return fail(SDD_ERR_INVALID_ARG, "NULL argument");
    if (bytes < sizeof(CheckpointHeader))
        return fail(SDD_ERR_INVALID_ARG, "not a checkpoint (too short)");
    CheckpointHeader h;
    memcpy(&h, host, sizeof(h));
    if (h.magic != kCheckpointMagic || h.version != 2 || h.slot_bytes != sizeof(Slot))
        return fail(SDD_ERR_INVALID_ARG, "not a checkpoint of this library");
    if (h.n != (uint64_t)p->n || h.n_mc != (uint64_t)p->n_mc || h.plan_hash != plan_hash(p))
        return fail(SDD_ERR_INVALID_ARG, "the checkpoint belongs to another plan");
    if (h.items_done > h.items_total ||
        bytes < sizeof(CheckpointHeader) + h.items_done * sizeof(Slot))
        return fail(SDD_ERR_INVALID_ARG, "checkpoint truncated");
    int rc = check_device(p);
    if (rc) return rc;
    if ((rc = validate_mc(&h.mc))) return rc;
    cudaStream_t stream = as_stream(stream_);
    McArgs a;
    bool few = false;
    if ((rc = mc_args(p, &h.mc, nullptr, nullptr, nullptr, a, few, stream))) return rc;
    if (a.total_items != h.items_total)
        return fail(SDD_ERR_INVALID_ARG, "the checkpoint's work-item count differs from the plan's");
    if (h.items_done)
        SDD_CUDA(cudaMemcpyAsync(p->d_slots, static_cast<const unsigned char*>(host) + sizeof(h),
                                 h.items_done * sizeof(Slot), cudaMemcpyHostToDevice, stream));
    SDD_CUDA(cudaStreamSynchronize(stream));
    p->items_valid = false;                      // the slots hold the checkpoint's items
    p->resume_active = true;
    p->resume_mc = h.mc;
    p->resume_next = h.items_done;
    p->resume_total = h.items_total;
    p->last_stream = stream;
    return SDD_OK;
}

int sdd_plan_last_mc_stats(sdd_plan* p, sdd_mc_stats* stats)
{
    clear_error();
    if (!p || !stats) return fail(SDD_ERR_INVALID_ARG, "NULL argument");
    if (!p->have_mc) return fail(SDD_ERR_INVALID_ARG, "no Monte Carlo call on this plan yet");
    int rc = check_device(p);
    if (rc) return rc;
    if (!p->mc_done)
        return fail(SDD_ERR_INVALID_ARG,
                    "this plan's last Monte Carlo run was part of a batch: use sdd_batch_plan_stats");
    // wait for this plan's last Monte Carlo call only, not for later work on its stream
    SDD_CUDA(cudaEventSynchronize(p->mc_done));
    McStatsDev s;
    SDD_CUDA(cudaMemcpy(&s, p->d_stats, sizeof(s), cudaMemcpyDeviceToHost));
    return stats_from_dev(s, p->last_paths * (uint64_t)p->n_mc, stats);
}

int sdd_subdomain_solve(sdd_plan* p, const double* iface, const sdd_solve_params* sp, double* mesh,
                        sdd_solve_stats* stats, void* stream_)
{
    NvtxRange nvtx_range("sdd_subdomain_solve");
    clear_error();
    if (!p || !mesh) return fail(SDD_ERR_INVALID_ARG, "NULL argument");
    if (!iface && p->n_nodes > 0) return fail(SDD_ERR_INVALID_ARG, "iface is NULL");
    int rc = check_device(p);
    if (rc) return rc;
    cudaStream_t stream = as_stream(stream_);
    const size_t ibytes = (size_t)p->n_nodes * 2 * sizeof(double);
    const double* iface_dev = iface;
    if (iface && !is_device_ptr(iface)) {
        if ((rc = ensure_mc_buffers(p, 0, stream))) return rc;
        SDD_CUDA(cudaMemcpyAsync(p->d_mean, iface, ibytes, cudaMemcpyHostToDevice, stream));
        iface_dev = p->d_mean;
    }
    if ((rc = run_solve(p, iface_dev, sp, stream))) return rc;
    const size_t mbytes = (size_t)p->n * p->n * 2 * sizeof(double);
    if (is_device_ptr(mesh)) {
        SDD_CUDA(cudaMemcpyAsync(mesh, p->d_u, mbytes, cudaMemcpyDeviceToDevice, stream));
    } else {
        SDD_CUDA(cudaMemcpyAsync(mesh, p->d_u, mbytes, cudaMemcpyDeviceToHost, stream));
        SDD_CUDA(cudaStreamSynchronize(stream));
    }
    if (stats) return read_solve_stats(p, stats, stream);
    return SDD_OK;
}

int sdd_mesh_generate(sdd_plan* p, const sdd_mc_params* mc, const sdd_solve_params* sp,
                      double* mesh, double* iface_mean, double* iface_stderr,
                      sdd_mc_stats* mc_stats, sdd_solve_stats* solve_stats, void* stream_)
{
    NvtxRange nvtx_range("sdd_mesh_generate");
    clear_error();
    if (!p || !mesh) return fail(SDD_ERR_INVALID_ARG, "NULL argument");
    int rc = check_device(p);
    if (rc) return rc;
    if ((rc = validate_solve(sp))) return rc;
    cudaStream_t stream = as_stream(stream_);
    if ((rc = run_mc(p, mc, nullptr, nullptr, nullptr, stream))) return rc;
    if ((rc = run_solve(p, p->d_mean, sp, stream))) return rc;
    const size_t mbytes = (size_t)p->n * p->n * 2 * sizeof(double);
    const size_t ibytes = (size_t)p->n_nodes * 2 * sizeof(double);
    bool host = false;
    if (is_device_ptr(mesh)) {
        SDD_CUDA(cudaMemcpyAsync(mesh, p->d_u, mbytes, cudaMemcpyDeviceToDevice, stream));
    } else {
        SDD_CUDA(cudaMemcpyAsync(mesh, p->d_u, mbytes, cudaMemcpyDeviceToHost, stream));
        host = true;
    }
    if (iface_mean && ibytes) {
        const bool d = is_device_ptr(iface_mean);
        SDD_CUDA(cudaMemcpyAsync(iface_mean, p->d_mean, ibytes,
                                 d ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, stream));
        host = host || !d;
    }
    if (iface_stderr && ibytes) {
        const bool d = is_device_ptr(iface_stderr);
        SDD_CUDA(cudaMemcpyAsync(iface_stderr, p->d_stderr, ibytes,
                                 d ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, stream));
        host = host || !d;
    }
    if (mc_stats && (rc = read_mc_stats(p, mc_stats, stream))) return rc;
    if (solve_stats) return read_solve_stats(p, solve_stats, stream);
    if (host) SDD_CUDA(cudaStreamSynchronize(stream));
    return SDD_OK;
}

void sdd_plan_destroy(sdd_plan* p)
{
    if (!p) return;
    // stream-ordered after the plan's last work; no device synchronisation
    const cudaStream_t fs = p->have_mc || p->last_stream ? p->last_stream : setup_stream();
    dev_free(p->d_nodes, fs);
    dev_free(p->d_edges, fs);
    dev_free(p->d_tab64, fs);
    dev_free(p->d_cell32, fs);
    dev_free(p->d_queue, fs);
    dev_free(p->d_slots, fs);
    dev_free(p->d_sums, fs);
    dev_free(p->d_mean, fs);
    dev_free(p->d_stderr, fs);
    dev_free(p->d_stats, fs);
    dev_free(p->d_u, fs);
    dev_free(p->d_cx, fs);
    dev_free(p->d_cy, fs);
    dev_free(p->d_cxf, fs);
    dev_free(p->d_cyf, fs);
    dev_free(p->d_work, fs);
    dev_free(p->d_mg, fs);
    dev_free(p->d_subs, fs);
    dev_free(p->d_substats, fs);
    dev_free(p->d_mc_nodes, fs);
    dev_free(p->d_mc_ids, fs);
    dev_free(p->d_interp, fs);
    dev_free(p->d_quality, fs);
    if (p->mc_done) cudaEventDestroy(p->mc_done);
    delete p;
}

const char* sdd_last_error(void) { return g_error.c_str(); }

int sdd_kernel_launches(uint64_t* count)
{
    if (!count) return fail(SDD_ERR_INVALID_ARG, "count is NULL");
    *count = g_launches.load(std::memory_order_relaxed);
    return SDD_OK;
}

int sdd_plan_set_placement(sdd_plan* p, int mode, int k)
{
    clear_error();
    if (!p) return fail(SDD_ERR_INVALID_ARG, "plan is NULL");
    if (mode != SDD_PLACE_ALL && mode != SDD_PLACE_EQUISPACED && mode != SDD_PLACE_EXTREMA)
        return fail(SDD_ERR_INVALID_ARG, "unknown placement mode");
    if (mode == SDD_PLACE_EQUISPACED && (k < 1 || k > p->n - 2))
        return fail(SDD_ERR_INVALID_ARG, "EQUISPACED needs 1 <= k <= n-2");
    int rc = check_device(p);
    if (rc) return rc;
    std::vector<uint8_t> mask = placement_mask(p, mode, k);
    std::vector<int32_t> sub;
    std::vector<uint32_t> ids;
    for (int64_t q = 0; q < p->n_nodes; ++q)
        if (mask[q]) {
            sub.push_back(p->h_nodes[2 * q]);
            sub.push_back(p->h_nodes[2 * q + 1]);
            ids.push_back((uint32_t)q);
        }
    const cudaStream_t ss = setup_stream();
    // the old placement's buffers may still be read by queued work
    const cudaStream_t fs = p->last_stream ? p->last_stream : ss;
    dev_free(p->d_mc_nodes, fs);
    dev_free(p->d_mc_ids, fs);
    dev_free(p->d_interp, fs);
    p->h_interp.clear();
    p->place_mode = mode;
    p->h_mask = mask;
    p->n_mc = (int64_t)ids.size();
    p->items_valid = false;                             // other Monte Carlo nodes
    if (p->n_mc == p->n_nodes) return SDD_OK;           // every node: the plain path
    if ((rc = ensure_mc_buffers(p, 0, ss))) return rc;
    std::vector<InterpEntry> ent = interp_entries(p, mask);
    for (InterpEntry& e : ent) {
        e.mean = p->d_mean;
        e.se = p->d_stderr;
    }
    AllocOn on(ss);
    if ((rc = dev_alloc(&p->d_mc_nodes, std::max<size_t>(ids.size(), 1))) ||
        (rc = dev_alloc(&p->d_mc_ids, std::max<size_t>(ids.size(), 1))) ||
        (rc = dev_alloc(&p->d_interp, std::max<size_t>(ent.size(), 1))))
        return rc;
    if (!ids.empty()) {
        SDD_CUDA(cudaMemcpyAsync(p->d_mc_nodes, sub.data(), sub.size() * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, ss));
        SDD_CUDA(cudaMemcpyAsync(p->d_mc_ids, ids.data(), ids.size() * sizeof(uint32_t),
                                 cudaMemcpyHostToDevice, ss));
    }
    if (!ent.empty())
        SDD_CUDA(cudaMemcpyAsync(p->d_interp, ent.data(), ent.size() * sizeof(InterpEntry),
                                 cudaMemcpyHostToDevice, ss));
    SDD_CUDA(cudaStreamSynchronize(ss));
    p->h_interp = std::move(ent);
    return SDD_OK;
}

int sdd_plan_placement(const sdd_plan* p, uint8_t* mask, int64_t* n_mc)
{
    clear_error();
    if (!p) return fail(SDD_ERR_INVALID_ARG, "plan is NULL");
    if (mask) std::copy(p->h_mask.begin(), p->h_mask.end(), mask);
    if (n_mc) *n_mc = p->n_mc;
    return SDD_OK;
}

int sdd_mesh_quality(sdd_plan* p, const double* mesh, const double* ref, sdd_quality* out,
                     void* stream_)
{
    NvtxRange nvtx_range("sdd_mesh_quality");
    clear_error();
    if (!p || !mesh || !out) return fail(SDD_ERR_INVALID_ARG, "NULL argument");
    int rc = check_device(p);
    if (rc) return rc;
    cudaStream_t stream = as_stream(stream_);
    const size_t bytes = (size_t)p->n * p->n * 2 * sizeof(double);
    double* tmp = nullptr;                       // device copies of host meshes
    const double* dm = mesh;
    const double* dr = ref;
    {
        AllocOn on(stream);
        const bool hm = !is_device_ptr(mesh), hr = ref && !is_device_ptr(ref);
        if (hm || hr) {
            if ((rc = dev_alloc(&tmp, (hm ? 2 : 0) * (size_t)p->n * p->n + (hr ? 2 : 0) * (size_t)p->n * p->n)))
                return rc;
            double* q = tmp;
            if (hm) {
                SDD_CUDA(cudaMemcpyAsync(q, mesh, bytes, cudaMemcpyHostToDevice, stream));
                dm = q;
                q += 2 * (size_t)p->n * p->n;
            }
            if (hr) {
                SDD_CUDA(cudaMemcpyAsync(q, ref, bytes, cudaMemcpyHostToDevice, stream));
                dr = q;
            }
        }
        if (!p->d_quality && (rc = dev_alloc(&p->d_quality, 1))) return rc;
    }
    rc = launch_quality(p->n, p->dens.family, p->dens.params, p->d_tab64, p->dens.tn, dm, dr,
                        p->d_quality, stream);
    if (rc) return rc;
    QualityDev q;
    SDD_CUDA(cudaMemcpyAsync(&q, p->d_quality, sizeof(q), cudaMemcpyDeviceToHost, stream));
    if (tmp) dev_free(tmp, stream);
    SDD_CUDA(cudaStreamSynchronize(stream));
    const double cells = (double)(p->n - 1) * (p->n - 1);
    auto dbl = [](unsigned long long b) { double d; memcpy(&d, &b, sizeof(d)); return d; };
    out->q_max = dbl(q.q_max_bits);
    out->folds = (int64_t)q.folds;
    out->q_mean = q.q_sum / std::max(cells - (double)q.folds, 1.0);
    out->ref_q_max = ref ? dbl(q.q_ref_max_bits) : 0.0;
    out->ref_folds = ref ? (int64_t)q.ref_folds : 0;
    out->ref_q_mean = ref ? q.q_ref_sum / std::max(cells - (double)q.ref_folds, 1.0) : 0.0;
    out->r_max = ref && out->q_max > 0 ? out->ref_q_max / out->q_max : 0.0;
    out->r_mean = ref && out->q_mean > 0 ? out->ref_q_mean / out->q_mean : 0.0;
    out->l_inf = ref ? dbl(q.l_inf_bits) : 0.0;
    return SDD_OK;
}

// Smoothing with the lines marked in `hold` (n bytes: bit 0 column, bit 1
// row; empty: none) held fixed besides the boundary.
static int smooth_mesh(sdd_plan* p, double* mesh, int steps, double dt, double k,
                       const std::vector<uint8_t>& hold, void* stream_)
{
    if (!p || !mesh) return fail(SDD_ERR_INVALID_ARG, "NULL argument");
    if (steps < 0) return fail(SDD_ERR_INVALID_ARG, "steps must be >= 0");
    if (!(dt > 0.0) || !std::isfinite(dt) || !(k > 0.0) || !std::isfinite(k))
        return fail(SDD_ERR_INVALID_ARG, "dt and k must be positive and finite");
    const double h = 1.0 / (double)(p->n - 1);
    if (dt / (h * h) > 0.25)
        return fail(SDD_ERR_INVALID_ARG, "dt (n-1)^2 = " + std::to_string(dt / (h * h)) +
                                             " exceeds 1/4: the FTCS step would be unstable");
    int rc = check_device(p);
    if (rc) return rc;
    if (steps == 0) return SDD_OK;
    cudaStream_t stream = as_stream(stream_);
    const size_t count = 2 * (size_t)p->n * p->n;            // doubles of one mesh
    const bool host = !is_device_ptr(mesh);
    double* tmp = nullptr;
    {
        AllocOn on(stream);
        if ((rc = dev_alloc(&tmp, (host ? 2 : 1) * count))) return rc;
    }
    double* u = host ? tmp + count : mesh;
    if (host)
        SDD_CUDA(cudaMemcpyAsync(u, mesh, count * sizeof(double), cudaMemcpyHostToDevice, stream));
    uint8_t* d_hold = nullptr;
    if (!hold.empty()) {
        {
            AllocOn on(stream);
            if ((rc = dev_alloc(&d_hold, hold.size()))) {
                dev_free(tmp, stream);
                return rc;
            }
        }
        // pageable source: the copy has taken the bytes when the call returns
        SDD_CUDA(cudaMemcpyAsync(d_hold, hold.data(), hold.size(), cudaMemcpyHostToDevice, stream));
    }
    rc = launch_smooth(p->n, u, tmp, steps, dt, k, d_hold, stream);
    if (d_hold) dev_free(d_hold, stream);
    if (rc) {
        dev_free(tmp, stream);
        return rc;
    }
    if (host) {
        SDD_CUDA(cudaMemcpyAsync(mesh, u, count * sizeof(double), cudaMemcpyDeviceToHost, stream));
        dev_free(tmp, stream);
        SDD_CUDA(cudaStreamSynchronize(stream));
    } else {
        dev_free(tmp, stream);
    }
    return SDD_OK;
}

int sdd_mesh_smooth(sdd_plan* p, double* mesh, int steps, double dt, double k, void* stream_)
{
    NvtxRange nvtx_range("sdd_mesh_smooth");
    clear_error();
    return smooth_mesh(p, mesh, steps, dt, k, {}, stream_);
}

// Lines bounding the blocks smoothed separately along one axis: the plan's
// interface lines, or (shifted) the midlines floor((a + b) / 2) of the blocks
// [a, b] between consecutive lines of 0, the interfaces and n - 1.
static std::vector<int> smoothing_lines(int n, const std::vector<int>& iface, bool shifted)
{
    if (!shifted) return iface;
    std::vector<int> X{0};
    X.insert(X.end(), iface.begin(), iface.end());
    X.push_back(n - 1);
    std::vector<int> mid;
    for (size_t a = 0; a + 1 < X.size(); ++a) mid.push_back((X[a] + X[a + 1]) / 2);
    return mid;
}

int sdd_mesh_smooth_subdomains(sdd_plan* p, double* mesh, int steps, double dt, double k,
                               int shifted, void* stream_)
{
    NvtxRange nvtx_range("sdd_mesh_smooth_subdomains");
    clear_error();
    if (!p) return fail(SDD_ERR_INVALID_ARG, "NULL argument");
    if (shifted != 0 && shifted != 1) return fail(SDD_ERR_INVALID_ARG, "shifted must be 0 or 1");
    std::vector<uint8_t> hold((size_t)p->n, 0);
    for (int i : smoothing_lines(p->n, p->ix, shifted != 0)) hold[(size_t)i] |= 1u;
    for (int j : smoothing_lines(p->n, p->iy, shifted != 0)) hold[(size_t)j] |= 2u;
    return smooth_mesh(p, mesh, steps, dt, k, hold, stream_);
}

int sdd_batch_create(sdd_plan* const* plans, int n_plans, const sdd_mc_params* mc,
                     const sdd_solve_params* sp, sdd_batch** out)
{
    NvtxRange nvtx_range("sdd_batch_create");
    clear_error();
    if (!out) return fail(SDD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!plans || !mc || !sp || n_plans <= 0)
        return fail(SDD_ERR_INVALID_ARG, "plans, mc and sp must hold n_plans > 0 entries");
    int rc;
    for (int i = 0; i < n_plans; ++i) {
        if (!plans[i]) return fail(SDD_ERR_INVALID_ARG, "NULL plan in batch");
        if ((rc = check_device(plans[i]))) return rc;
        if ((rc = validate_mc(&mc[i]))) return rc;
        if ((rc = validate_solve(&sp[i]))) return rc;
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return fail(SDD_ERR_INVALID_ARG, "a plan appears twice in a batch");
    }
    sdd_batch* b = new (std::nothrow) sdd_batch();
    if (!b) return fail(SDD_ERR_OOM, "host allocation failed");
    cudaGetDevice(&b->device);
    b->plans.assign(plans, plans + n_plans);
    b->plan_slot.assign(n_plans, -1);
    for (int i = 0; i < n_plans; ++i) b->plan_paths.push_back(mc[i].paths_per_node);

    // per-plan device buffers (outputs, solve buffers, edge coefficients) and
    // the batch's records are set up on the library's set-up stream, which is
    // synchronised (alone) before the batch is returned
    const cudaStream_t ss = setup_stream();
    AllocOn on(ss);
    for (int i = 0; i < n_plans; ++i) {
        if ((rc = ensure_mc_buffers(plans[i], 0, ss)) || (rc = alloc_solve_buffers(plans[i], ss))) {
            batch_free(b);
            return rc;
        }
    }
    // group meshes by (precision, kernel class); records in group order
    std::vector<std::pair<int, int>> key(n_plans);
    for (int i = 0; i < n_plans; ++i) {
        const int nb = plans[i]->dens.family == SDD_FAMILY_BUMPS ? (int)plans[i]->dens.params[0] : 0;
        key[i] = {mc[i].precision, mesh_kernel_class(plans[i]->dens.family, nb, mc[i].stepper,
                                                       mc[i].exit_test)};
    }
    std::vector<int> order(n_plans);
    for (int i = 0; i < n_plans; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return key[x] < key[y]; });

    std::vector<MeshDev> recs(n_plans);
    std::vector<uint64_t> offs;
    uint64_t slot_total = 0;
    struct GInfo { int precision, kc, first, count; size_t item_off, node_off; uint64_t items, nodes, slot_base; };
    std::vector<GInfo> gi;
    for (int k = 0; k < n_plans;) {
        int e = k;
        while (e < n_plans && key[order[e]] == key[order[k]]) ++e;
        GInfo g{key[order[k]].first, key[order[k]].second, k, e - k, 0, 0, 0, 0, slot_total};
        g.item_off = offs.size();
        uint64_t it = 0;
        for (int q = k; q < e; ++q) {
            const int i = order[q];
            MeshDev& m = recs[q];
            mesh_record(plans[i], &mc[i], m);
            if (plans[i]->n_mc < plans[i]->n_nodes) {          // few-point interface
                m.n_nodes = plans[i]->n_mc;
                if (!mc[i].chunk) {
                    m.chunk = auto_chunk(mc[i].paths_per_node, plans[i]->n_mc);
                    m.chunks_per_node = (uint32_t)((mc[i].paths_per_node + m.chunk - 1) / m.chunk);
                }
            }
            if (mc[i].path_begin) {
                if ((rc = check_continuation(plans[i], &mc[i], m.n_nodes))) {
                    batch_free(b);
                    return rc;
                }
                b->seeds.push_back(SlotSeed{plans[i], plans[i]->items_run, plans[i]->d_slots,
                                            slot_total + it,
                                            mc[i].path_begin / m.chunk, m.chunks_per_node,
                                            (uint64_t)m.n_nodes});
            }
            m.item_begin = it;
            offs.push_back(it);
            it += (uint64_t)m.n_nodes * m.chunks_per_node;
            b->plan_slot[i] = q;
        }
        offs.push_back(it);
        g.items = it;
        g.node_off = offs.size();
        uint64_t nd = 0;
        for (int q = k; q < e; ++q) {
            recs[q].node_begin = nd;
            offs.push_back(nd);
            nd += (uint64_t)recs[q].n_nodes;
        }
        offs.push_back(nd);
        g.nodes = nd;
        slot_total += it;
        gi.push_back(g);
        k = e;
    }
    // solve records, fill records, subdomain list
    std::vector<SolveMeshDev> sm(n_plans);
    std::vector<FillDev> fill(n_plans);
    std::vector<uint64_t> fill_off(n_plans + 1, 0);
    std::vector<SubDev> subs;
    for (int i = 0; i < n_plans; ++i) {
        sdd_plan* p = plans[i];
        SolveMeshDev& r = sm[i];
        memset(&r, 0, sizeof(r));
        r.n = p->n;
        r.solver = sp[i].solver;
        b->solver_mask |= solver_bit(sp[i].solver);
        b->solve_threads = std::max(b->solve_threads, (int)sp[i].block_threads);
        r.max_iter = sp[i].max_iter > 0 ? sp[i].max_iter : (sp[i].solver == SDD_SOLVER_SOR ? 200000 : 20000);
        r.tol = sp[i].tol;
        r.omega = sp[i].omega;
        r.u = p->d_u;
        r.cx = p->d_cx;
        r.cy = p->d_cy;
        r.cxf = p->d_cxf;
        r.cyf = p->d_cyf;
        r.work = p->d_work;
        r.mg = p->d_mg;
        FillDev& f = fill[i];
        memset(&f, 0, sizeof(f));
        f.n = p->n;
        f.n_nodes = p->n_nodes;
        f.edges = p->d_edges;
        f.nodes = p->d_nodes;
        f.iface = p->d_mean;
        f.u = p->d_u;
        fill_off[i + 1] = fill_off[i] + 4 * (uint64_t)p->n + (uint64_t)p->n_nodes;
        b->sub_begin.push_back((int)subs.size());
        for (SubDev d : p->h_subs) {
            d.mesh = i;
            d.slot += b->sub_begin.back();      // stats in plan order, plan by plan
            subs.push_back(d);
        }
    }
    b->n_subs = (int)subs.size();
    b->fill_total = fill_off[n_plans];
    sort_largest_first(subs);

    const size_t ng = gi.size();
    if ((rc = dev_alloc(&b->d_meshes, recs.size())) || (rc = dev_alloc(&b->d_offs, offs.size())) ||
        (rc = dev_alloc(&b->d_slots, (size_t)std::max<uint64_t>(slot_total, 1))) ||
        (rc = dev_alloc(&b->d_queues, ng)) || (rc = dev_alloc(&b->d_stats, (size_t)n_plans)) ||
        (rc = dev_alloc(&b->d_fill, (size_t)n_plans)) ||
        (rc = dev_alloc(&b->d_fill_off, (size_t)n_plans + 1)) ||
        (rc = dev_alloc(&b->d_smesh, (size_t)n_plans)) ||
        (rc = dev_alloc(&b->d_subs, std::max<size_t>(subs.size(), 1))) ||
        (rc = dev_alloc(&b->d_substats, std::max<size_t>(subs.size(), 1)))) {
        batch_free(b);
        return rc;
    }
    // outputs of each record: the plan's own buffers; stats per plan
    std::vector<InterpEntry> interp;
    for (int i = 0; i < n_plans; ++i) {
        MeshDev& m = recs[b->plan_slot[i]];
        m.sums = plans[i]->d_sums;
        m.mean = plans[i]->d_mean;
        m.stderr_ = plans[i]->d_stderr;
        m.stats = b->d_stats + i;
        if (plans[i]->n_mc < plans[i]->n_nodes) {
            m.nodes = plans[i]->d_mc_nodes;
            m.node_ids = plans[i]->d_mc_ids;
            interp.insert(interp.end(), plans[i]->h_interp.begin(), plans[i]->h_interp.end());
        }
    }
    b->n_interp = (int64_t)interp.size();
    if (!interp.empty()) {
        if ((rc = dev_alloc(&b->d_interp, interp.size()))) {
            batch_free(b);
            return rc;
        }
        cudaError_t ie = cudaMemcpyAsync(b->d_interp, interp.data(), interp.size() * sizeof(InterpEntry),
                                         cudaMemcpyHostToDevice, ss);
        if (ie != cudaSuccess) {
            rc = cuda_status(ie, "cudaMemcpyAsync(batch interpolation)");
            batch_free(b);
            return rc;
        }
    }
    const auto h2d = cudaMemcpyHostToDevice;
    cudaError_t ce = cudaMemcpyAsync(b->d_meshes, recs.data(), recs.size() * sizeof(MeshDev), h2d, ss);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(b->d_offs, offs.data(), offs.size() * sizeof(uint64_t), h2d, ss);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(b->d_fill, fill.data(), fill.size() * sizeof(FillDev), h2d, ss);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(b->d_fill_off, fill_off.data(), fill_off.size() * sizeof(uint64_t), h2d, ss);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(b->d_smesh, sm.data(), sm.size() * sizeof(SolveMeshDev), h2d, ss);
    if (ce == cudaSuccess && !subs.empty()) ce = cudaMemcpyAsync(b->d_subs, subs.data(), subs.size() * sizeof(SubDev), h2d, ss);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(ss);
    if (ce != cudaSuccess) {
        rc = cuda_status(ce, "cudaMemcpy(batch records)");
        batch_free(b);
        return rc;
    }
    for (size_t k = 0; k < ng; ++k) {
        const GInfo& g = gi[k];
        McGroup G;
        memset(&G, 0, sizeof(G));
        G.precision = g.precision;
        G.kc = g.kc;
        if ((rc = mc_grid_blocks(g.precision, g.kc, false, &G.blocks, nullptr))) {
            batch_free(b);
            return rc;
        }
        McArgs& a = G.args;
        a.meshes = b->d_meshes + g.first;
        a.n_meshes = g.count;
        a.item_off = b->d_offs + g.item_off;
        a.node_off = b->d_offs + g.node_off;
        a.total_items = g.items;
        a.total_nodes = g.nodes;
        a.queue = b->d_queues + k;
        a.slots = b->d_slots + g.slot_base;
        b->groups.push_back(G);
    }
    *out = b;
    return SDD_OK;
}

int sdd_batch_run(sdd_batch* b, int use_graph, void* stream_)
{
    NvtxRange nvtx_range("sdd_batch_run");
    clear_error();
    if (!b) return fail(SDD_ERR_INVALID_ARG, "batch is NULL");
    int dev = -1;
    SDD_CUDA(cudaGetDevice(&dev));
    if (dev != b->device) return fail(SDD_ERR_INVALID_ARG, "batch belongs to another device");
    cudaStream_t stream = as_stream(stream_);
    int rc;
    if ((rc = check_seeds(b))) return rc;
    if (use_graph) {
        if (stream == nullptr)
            return fail(SDD_ERR_INVALID_ARG, "a graph launch needs a non-default stream");
        if (!b->graph_exec) {
            SDD_CUDA(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
            const uint64_t c0 = launches_now();
            rc = batch_enqueue(b, stream);
            b->graph_kernels = launches_now() - c0;
            count_launch(0 - b->graph_kernels);          // captured, not launched yet
            cudaGraph_t g = nullptr;
            cudaError_t ce = cudaStreamEndCapture(stream, &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            SDD_CUDA(ce);
            b->graph = g;
            SDD_CUDA(cudaGraphInstantiate(&b->graph_exec, b->graph, 0));
        }
        SDD_CUDA(cudaGraphLaunch(b->graph_exec, stream));
        count_launch(b->graph_kernels);
    } else {
        if ((rc = batch_enqueue(b, stream))) return rc;
    }
    for (size_t i = 0; i < b->plans.size(); ++i) {
        sdd_plan* p = b->plans[i];
        p->last_paths = b->plan_paths[i];
        p->have_mc = true;
        p->last_stream = stream;
        if (p->mc_done) {                        // the batch's stats live in the batch
            cudaEventDestroy(p->mc_done);
            p->mc_done = nullptr;
        }
    }
    b->last_stream = stream;
    b->ran = true;
    return SDD_OK;
}

int sdd_batch_run_phases(sdd_batch* b, int phases, void* stream_)
{
    NvtxRange nvtx_range("sdd_batch_run_phases");
    clear_error();
    if (!b) return fail(SDD_ERR_INVALID_ARG, "batch is NULL");
    if (phases < 1 || phases > 3) return fail(SDD_ERR_INVALID_ARG, "phases must be 1, 2 or 3");
    int dev = -1;
    SDD_CUDA(cudaGetDevice(&dev));
    if (dev != b->device) return fail(SDD_ERR_INVALID_ARG, "batch belongs to another device");
    cudaStream_t stream = as_stream(stream_);
    int rc = (phases & 1) ? check_seeds(b) : SDD_OK;
    if (rc) return rc;
    rc = batch_enqueue(b, stream, phases);
    if (rc) return rc;
    if (phases & 1) {
        for (size_t i = 0; i < b->plans.size(); ++i) {
            sdd_plan* p = b->plans[i];
            p->last_paths = b->plan_paths[i];
            p->have_mc = true;
            if (p->mc_done) {
                cudaEventDestroy(p->mc_done);
                p->mc_done = nullptr;
            }
        }
    }
    for (sdd_plan* p : b->plans) p->last_stream = stream;
    b->last_stream = stream;
    b->ran = true;
    return SDD_OK;
}

int sdd_batch_plan_stats(sdd_batch* b, int index, sdd_mc_stats* mc, sdd_solve_stats* solve)
{
    clear_error();
    if (!b || index < 0 || index >= (int)b->plans.size())
        return fail(SDD_ERR_INVALID_ARG, "bad batch or index");
    if (!b->ran) return fail(SDD_ERR_INVALID_ARG, "the batch has not run yet");
    SDD_CUDA(cudaStreamSynchronize(b->last_stream));
    sdd_plan* p = b->plans[index];
    int rc = SDD_OK;
    if (mc) {
        McStatsDev s;
        SDD_CUDA(cudaMemcpy(&s, b->d_stats + index, sizeof(s), cudaMemcpyDeviceToHost));
        if ((rc = stats_from_dev(s, b->plan_paths[index] * (uint64_t)p->n_mc, mc))) return rc;
    }
    if (solve) {
        const int nsub = (int)p->h_subs.size();
        std::vector<SubStat> st(nsub);
        if (nsub)
            SDD_CUDA(cudaMemcpy(st.data(), b->d_substats + b->sub_begin[index],
                                nsub * sizeof(SubStat), cudaMemcpyDeviceToHost));
        solve->subdomains = nsub;
        solve->converged = 0;
        solve->max_iterations = 0;
        solve->max_rel_residual = 0.0;
        solve->node_iterations = 0.0;
        for (const SubStat& x : st) {
            solve->converged += x.converged;
            solve->max_iterations = std::max(solve->max_iterations, x.iterations);
            solve->max_rel_residual = std::max(solve->max_rel_residual, x.rel_residual);
        }
        for (const SubDev& d : p->h_subs)
            solve->node_iterations += (double)st[d.slot].iterations * interior_nodes(d);
        if (solve->converged != solve->subdomains)
            return fail(SDD_ERR_NOT_CONVERGED, "a subdomain did not reach the tolerance");
    }
    return SDD_OK;
}

void sdd_batch_destroy(sdd_batch* b)
{
    if (!b) return;
    batch_free(b);                 // stream-ordered after the batch's last run
}

int sdd_plan_results(sdd_plan* p, double* mesh, double* mean, double* stderr_, void* stream_)
{
    clear_error();
    if (!p) return fail(SDD_ERR_INVALID_ARG, "plan is NULL");
    int rc = check_device(p);
    if (rc) return rc;
    cudaStream_t stream = as_stream(stream_);
    bool host = false;
    const size_t mbytes = (size_t)p->n * p->n * 2 * sizeof(double);
    const size_t ibytes = (size_t)p->n_nodes * 2 * sizeof(double);
    if (mesh) {
        if (!p->d_u) return fail(SDD_ERR_INVALID_ARG, "no mesh has been generated on this plan");
        const bool d = is_device_ptr(mesh);
        SDD_CUDA(cudaMemcpyAsync(mesh, p->d_u, mbytes, d ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, stream));
        host = host || !d;
    }
    if ((mean || stderr_) && !p->have_mc)
        return fail(SDD_ERR_INVALID_ARG, "no Monte Carlo call on this plan yet");
    if (mean && ibytes) {
        const bool d = is_device_ptr(mean);
        SDD_CUDA(cudaMemcpyAsync(mean, p->d_mean, ibytes, d ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, stream));
        host = host || !d;
    }
    if (stderr_ && ibytes) {
        const bool d = is_device_ptr(stderr_);
        SDD_CUDA(cudaMemcpyAsync(stderr_, p->d_stderr, ibytes, d ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, stream));
        host = host || !d;
    }
    if (host) SDD_CUDA(cudaStreamSynchronize(stream));
    return SDD_OK;
}

}  // extern "C"

// ------------------------------------------- allocation-free Monte Carlo --
// Some callers cannot allocate device memory: code that runs where the
// allocator is owned by someone else (a framework's caching allocator, an
// embedded runtime with a fixed memory budget) or where a cudaMalloc would
// synchronise or fail at the wrong moment.  For them sdd_interface_mc_static
// runs the same path kernel and reduction as sdd_interface_mc, with every byte
// of its scratch (work counter, counters, per-work-item sums) in this
// file-scope device array.  Every GPU that loads the library holds the array
// until the process exits.
namespace {

constexpr size_t kStaticScratchBytes = size_t(8) << 20;            // 8 MiB
constexpr size_t kStaticHeadBytes = 512;                           // counter + stats
constexpr uint64_t kStaticMaxItems = (kStaticScratchBytes - kStaticHeadBytes) / sizeof(Slot);

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Driver calls reached through the runtime's entry-point lookup, so that the
// library does not link libcuda (it still loads on machines without a GPU).
using MemRangeFn = CUresult (*)(CUdeviceptr*, size_t*, CUdeviceptr);
using CtxCurrentFn = CUresult (*)(CUcontext*);
using CtxIdFn = CUresult (*)(CUcontext, unsigned long long*);

template <typename F>
int driver_fn(const char* name, F* out)
{
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion(name, &f, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !f) {
        cudaGetLastError();
        return fail(SDD_ERR_CUDA, std::string("driver entry point ") + name + " not available");
    }
    *out = reinterpret_cast<F>(f);
    return SDD_OK;
}

struct StaticState {
    void* ptr = nullptr;              // device address of the array in this context
    unsigned long long ctx = 0;       // id of the context it was looked up in
    uint64_t paths = 0;               // paths of the last call, all nodes (statistics)
};
std::mutex g_static_mu;
StaticState g_static[64];

// Device address of the array for the current device: looked up with that
// device current on the first call, and again whenever the device's current
// context is another one than at the last lookup (after a cudaDeviceReset
// the array lives at a new address).
int static_scratch(void** out, int* dev_out)
{
    int dev = -1;
    SDD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(SDD_ERR_NO_DEVICE, "device index out of range");
    SDD_CUDA(cudaSetDevice(dev));                    // initialises the device's primary context
    static CtxCurrentFn ctx_current = nullptr;
    static CtxIdFn ctx_id = nullptr;
    std::lock_guard<std::mutex> lock(g_static_mu);
    int rc;
    if (!ctx_current && (rc = driver_fn("cuCtxGetCurrent", &ctx_current))) return rc;
    if (!ctx_id && (rc = driver_fn("cuCtxGetId", &ctx_id))) return rc;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (ctx_current(&ctx) != CUDA_SUCCESS || !ctx || ctx_id(ctx, &id) != CUDA_SUCCESS)
        return fail(SDD_ERR_CUDA, "no current CUDA context for the static scratch");
    StaticState& st = g_static[dev];
    if (!st.ptr || st.ctx != id) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(static scratch)");
        st.ptr = p;
        st.ctx = id;
    }
    *out = st.ptr;
    *dev_out = dev;
    return SDD_OK;
}

// A caller's buffer must be device (or managed) memory of the current device,
// aligned for its element type, and hold `bytes` bytes from `p` on within its
// allocation (cuMemGetAddressRange), so that no kernel of the call can read
// or write outside it.
int check_span(const void* p, size_t bytes, size_t align, int dev, const char* name)
{
    if (reinterpret_cast<uintptr_t>(p) % align)
        return fail(SDD_ERR_INVALID_ARG, std::string(name) + " must be aligned to " +
                                             std::to_string(align) + " bytes");
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) cudaGetLastError();
    if (e != cudaSuccess ||
        (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged))
        return fail(SDD_ERR_INVALID_ARG, std::string(name) + " must be device memory");
    if (at.type == cudaMemoryTypeDevice && at.device != dev)
        return fail(SDD_ERR_INVALID_ARG, std::string(name) + " is memory of another device");
    static MemRangeFn range = nullptr;
    int rc;
    {
        std::lock_guard<std::mutex> lock(g_static_mu);
        if (!range && (rc = driver_fn("cuMemGetAddressRange", &range))) return rc;
    }
    CUdeviceptr base = 0;
    size_t size = 0;
    if (range(&base, &size, (CUdeviceptr)reinterpret_cast<uintptr_t>(p)) != CUDA_SUCCESS)
        return fail(SDD_ERR_INVALID_ARG, std::string(name) + ": no device allocation holds it");
    const uint64_t have = (uint64_t)base + size - (uint64_t)reinterpret_cast<uintptr_t>(p);
    if (have < bytes)
        return fail(SDD_ERR_INVALID_ARG, std::string(name) + " needs " + std::to_string(bytes) +
                                             " bytes, its allocation holds " +
                                             std::to_string(have) + " from the pointer on");
    return SDD_OK;
}

}  // namespace

extern "C" int sdd_interface_mc_static(int n, const int32_t* nodes, int64_t n_nodes,
                                       const double* edges, const sdd_density* dens,
                                       const sdd_mc_params* mc, double* mean, double* stderr_,
                                       void* stream_)
{
    clear_error();
    if (n < 3 || n > 16385) return fail(SDD_ERR_INVALID_ARG, "n must be in [3, 16385]");
    if (n_nodes < 1) return fail(SDD_ERR_INVALID_ARG, "n_nodes must be >= 1");
    if (!nodes || !edges || !mean)
        return fail(SDD_ERR_INVALID_ARG, "nodes, edges and mean are required");
    int rc = validate_density(dens);
    if (rc) return rc;
    if (dens->family == SDD_FAMILY_TABLE)
        return fail(SDD_ERR_INVALID_ARG,
                    "the allocation-free entry point takes the analytic families only "
                    "(a TABLE density is copied to the device by a plan)");
    if ((rc = validate_mc(mc))) return rc;
    if (mc->path_begin)
        return fail(SDD_ERR_INVALID_ARG, "the allocation-free entry point takes path_begin = 0");
    // work-item size: the caller's, else the automatic one, raised (up to 8192
    // paths) until the work items fit the static array
    uint32_t chunk = mc->chunk ? (uint32_t)mc->chunk : auto_chunk(mc->paths_per_node, n_nodes);
    auto items_for = [&](uint32_t c) {
        return (uint64_t)n_nodes * ((mc->paths_per_node + c - 1) / c);
    };
    if (!mc->chunk)
        while (items_for(chunk) > kStaticMaxItems && chunk < 8192) chunk *= 2;
    chunk = std::min<uint32_t>(chunk, 8192);
    const uint64_t items = items_for(chunk);
    if (items > kStaticMaxItems)
        return fail(SDD_ERR_INVALID_ARG,
                    "too much work for the static scratch: n_nodes * ceil(N / chunk) = " +
                        std::to_string(items) + " work items, at most " +
                        std::to_string(kStaticMaxItems) + " fit in 8 MiB");
    void* base = nullptr;
    int dev = -1;
    if ((rc = static_scratch(&base, &dev))) return rc;
    const size_t node_bytes = (size_t)n_nodes * 2 * sizeof(double);
    if ((rc = check_span(nodes, (size_t)n_nodes * 2 * sizeof(int32_t), 8, dev, "nodes")) ||
        (rc = check_span(edges, (size_t)8 * n * sizeof(double), 8, dev, "edges")) ||
        (rc = check_span(mean, node_bytes, 8, dev, "mean")) ||
        (stderr_ && (rc = check_span(stderr_, node_bytes, 8, dev, "stderr_"))))
        return rc;
    unsigned char* b = static_cast<unsigned char*>(base);
    cudaStream_t stream = as_stream(stream_);

    McArgs a;
    memset(&a, 0, sizeof(a));
    MeshDev& m = a.single;
    m.n = n;
    m.family = dens->family;
    m.precision = mc->precision;
    m.key0 = (uint32_t)(mc->seed & 0xffffffffu);
    m.key1 = (uint32_t)(mc->seed >> 32);
    m.paths = (uint32_t)mc->paths_per_node;
    m.chunk = chunk;
    m.chunks_per_node = (uint32_t)((mc->paths_per_node + chunk - 1) / chunk);
    m.max_steps = (uint32_t)(mc->max_steps ? mc->max_steps : (uint64_t)std::ceil(2.0 / mc->dt));
    m.bridge = mc->exit_test == SDD_EXIT_BRIDGE ? 1 : 0;
    m.stepper = mc->stepper;
    m.n_nodes = n_nodes;
    m.dt = mc->dt;
    m.sqrt2dt = std::sqrt(2.0 * mc->dt);
    m.tie_delta = mc->tie_delta >= 0.0 ? mc->tie_delta : (mc->precision == SDD_FP64 ? 1e-11 : 0.0);
    m.nodes = reinterpret_cast<const int2*>(nodes);
    m.edges = edges;
    m.sums = nullptr;
    m.mean = mean;
    m.stderr_ = stderr_;
    m.stats = reinterpret_cast<McStatsDev*>(b + 256);
    sdd_density d = *dens;
    for (int q = d.n_params; q < SDD_MAX_PARAMS; ++q) d.params[q] = 0.0;
    fill_fp32_params(m, d);
    for (int r = 0; r < 10; ++r) {
        a.rk[2 * r] = m.key0 + (uint32_t)r * 0x9E3779B9u;
        a.rk[2 * r + 1] = m.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    a.meshes = nullptr;
    a.n_meshes = 1;
    a.total_items = items;
    a.total_nodes = (uint64_t)n_nodes;
    a.queue = reinterpret_cast<unsigned long long*>(b);          // zeroed by the launcher
    a.slots = reinterpret_cast<Slot*>(b + kStaticHeadBytes);     // written before read
    SDD_CUDA(cudaMemsetAsync(m.stats, 0, sizeof(McStatsDev), stream));
    rc = launch_mc(a, mc->precision, mesh_kernel_class(m.family, m.nb, m.stepper, mc->exit_test),
                   stream);
    if (rc == SDD_OK) {
        std::lock_guard<std::mutex> lock(g_static_mu);
        g_static[dev].paths = mc->paths_per_node * (uint64_t)n_nodes;   // paths of all nodes
    }
    return rc;
}

extern "C" int sdd_interface_mc_static_stats(sdd_mc_stats* stats, void* stream_)
{
    clear_error();
    if (!stats) return fail(SDD_ERR_INVALID_ARG, "stats is NULL");
    void* base = nullptr;
    int dev = -1;
    int rc = static_scratch(&base, &dev);
    if (rc) return rc;
    uint64_t paths;
    {
        std::lock_guard<std::mutex> lock(g_static_mu);
        paths = g_static[dev].paths;
    }
    if (!paths) return fail(SDD_ERR_INVALID_ARG, "no allocation-free Monte Carlo call on this device yet");
    McStatsDev h;
    cudaStream_t stream = as_stream(stream_);
    SDD_CUDA(cudaMemcpyAsync(&h, static_cast<unsigned char*>(base) + 256, sizeof(h),
                             cudaMemcpyDeviceToHost, stream));
    SDD_CUDA(cudaStreamSynchronize(stream));
    return stats_from_dev(h, paths, stats);
}
