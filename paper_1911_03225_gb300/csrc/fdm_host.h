// fdm_host.h -- host-side helpers shared by the single-instance and batch C ABIs:
// parameter validation, the loading law (Sec. 5.1), compensated sums, device buffers of a
// group, host<->device field copies, CUDA graphs of whole steps.
#pragma once
#include <cmath>
#include <cstring>
#include <vector>

#include "fdm_internal.h"

namespace fdm {

#define FDM_CK(x)                          \
    do {                                   \
        cudaError_t e_ = (x);              \
        if (e_ != cudaSuccess) {           \
            cudaGetLastError();            \
            return FDM_ERR_DEVICE;         \
        }                                  \
    } while (0)

inline bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

inline bool params_valid(const fdm_params* p) {
    if (!p) return false;
    if (!pow2_in(p->n1, 16, 4096) || !pow2_in(p->n2, 16, 4096)) return false;
    int nz = p->nz == 0 ? p->n1 : p->nz;
    if (nz < 1 || nz > 65536 || p->nh < 1 || p->nh > nz) return false;
    if (!(p->dx > 0.0) || !std::isfinite(p->dx)) return false;
    if (!(p->E > 0.0) || !(p->nu > -1.0 && p->nu < 0.5)) return false;
    if (p->velocity_mode != FDM_V_PRESCRIBED && p->velocity_mode != FDM_V_STRESS) return false;
    if (!std::isfinite(p->v0) || !std::isfinite(p->mobility) || !std::isfinite(p->tau_y)) return false;
    if (p->tau_y != 0.0 && !(p->beta > 0.0)) return false;
    if (!(p->theta >= 1.0 && p->theta <= 2.0)) return false;
    if (!(p->cfl > 0.0 && p->cfl <= 1.0)) return false;
    if (!std::isfinite(p->dt_max)) return false;
    if (p->loading_mode < FDM_LOAD_STRESS || p->loading_mode > FDM_LOAD_STRAIN_RATE) return false;
    if (!std::isfinite(p->sigma_bar13) || !std::isfinite(p->eps_bar13_0) || !std::isfinite(p->eps_bar13_rate))
        return false;
    if (p->time_level != FDM_T_MIDPOINT && p->time_level != FDM_T_LITERAL) return false;
    if (p->precision != FDM_FP64 && p->precision != FDM_MIXED && p->precision != FDM_DF64) return false;
    if (p->autotune != 0 && p->autotune != 1) return false;
    return true;
}

// launch shapes of a group, as reported by the C ABI
template <typename T>
inline void launch_config(const LaunchGeom& g, fdm_launch_config* c) {
    std::memset(c, 0, sizeof(*c));
    c->rows_per_block = g.R;
    c->cols_per_block = g.C;
    knp_shape_info<T>(g.knp_shape, &c->stencil_block_rows, &c->stencil_nodes, &c->stencil_min_blocks);
    c->tuned = g.tuned;
    for (int k = 0; k < kKernelsPerStep; ++k) c->kernel_us[k] = g.tuned ? g.kernel_us[k] : 0.0;
}

// the configurations the autotuner times (candidate i of each kernel, cycling)
template <typename T>
inline int launch_candidates(const fdm_params& p, fdm_launch_config* out, int max) {
    int Rs[8], Cs[8];
    const int nR = row_candidates<T>(p.n1, p.n2, Rs, 8), nC = col_candidates<T>(p.n1, p.n2, Cs, 8);
    if (nR == 0 || nC == 0) return 0;
    int n = nR > nC ? nR : nC;
    if (kKnpShapes > n) n = kKnpShapes;
    for (int i = 0; i < n && i < max; ++i)
        launch_config<T>(geometry<T>(p.n1, p.n2, Rs[i % nR], Cs[i % nC], i % kKnpShapes), &out[i]);
    return n;
}

// launch shapes from a configuration, if it names candidates of this grid and precision
template <typename T>
inline bool geometry_from_config(const fdm_params& p, const fdm_launch_config& c, LaunchGeom* g) {
    int Rs[8], Cs[8];
    const int nR = row_candidates<T>(p.n1, p.n2, Rs, 8), nC = col_candidates<T>(p.n1, p.n2, Cs, 8);
    bool r_ok = false, c_ok = false;
    for (int i = 0; i < nR; ++i) r_ok = r_ok || Rs[i] == c.rows_per_block;
    for (int i = 0; i < nC; ++i) c_ok = c_ok || Cs[i] == c.cols_per_block;
    int shape = -1;
    for (int k = 0; k < kKnpShapes && shape < 0; ++k) {
        int ty, npt, minb;
        knp_shape_info<T>(k, &ty, &npt, &minb);
        if (ty == c.stencil_block_rows && npt == c.stencil_nodes && minb == c.stencil_min_blocks) shape = k;
    }
    if (!r_ok || !c_ok || shape < 0) return false;
    *g = geometry<T>(p.n1, p.n2, c.rows_per_block, c.cols_per_block, shape);
    return true;
}

inline size_t elt_size(const fdm_params* p) { return p->precision == FDM_MIXED ? sizeof(float) : sizeof(double); }

inline int red_blocks_for(size_t n) {
    size_t b = (n + 255) / 256;
    if (b > 1024) b = 1024;
    return (int)b;
}

// macroscopic loading state (Sec. 3.1.2 sigma-hat(0); Sec. 5.1), same law as the kernels
inline void host_loading(const fdm_params& p, long long step, double t, double mean, double* eps, double* sig) {
    const double mu = p.E / (2.0 * (1.0 + p.nu));
    const double frac = (double)p.nh / (double)p.nz;
    if (p.loading_mode == FDM_LOAD_STRESS) {
        *sig = p.sigma_bar13;
        *eps = (p.sigma_bar13 + mu * frac * mean) / (2.0 * mu);
    } else if (p.loading_mode == FDM_LOAD_STRAIN_RAMP || p.loading_mode == FDM_LOAD_STRAIN_RATE) {
        *eps = p.eps_bar13_0 + p.eps_bar13_rate * (p.loading_mode == FDM_LOAD_STRAIN_RAMP ? (double)step : t);
        *sig = 2.0 * mu * (*eps) - mu * frac * mean;
    } else {
        *eps = 0.5 * frac * mean;
        *sig = 0.0;
    }
}

// Neumaier sum of host values
inline double ksum(const double* x, size_t n) {
    double s = 0.0, c = 0.0;
    for (size_t i = 0; i < n; ++i) {
        double t = s + x[i];
        c += (std::fabs(s) >= std::fabs(x[i])) ? (s - t) + x[i] : (x[i] - t) + s;
        s = t;
    }
    return s + c;
}

// Bytes of the scalars' slot at the head of a group's pinned readout buffer (16-aligned).
constexpr size_t kInfoScalarBytes = (sizeof(fdm_dev_scalars) + 15) / 16 * 16;

// Test hook (fdm_debug_fail_allocation): allocations left before one fails, or -1.
extern int g_fail_alloc_countdown;
inline bool injected_alloc_failure() {
    if (g_fail_alloc_countdown < 0) return false;
    if (g_fail_alloc_countdown-- == 0) return true;
    return false;
}

// Device memory (and small pinned host buffers) owned by one handle or batch; freed together.
struct Arena {
    std::vector<void*> owned;
    std::vector<void*> owned_host;
    fdm_status alloc_host(void** ptr, size_t bytes) {
        *ptr = nullptr;
        if (injected_alloc_failure()) return FDM_ERR_OOM;
        cudaError_t e = cudaMallocHost(ptr, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            *ptr = nullptr;
            return e == cudaErrorMemoryAllocation ? FDM_ERR_OOM : FDM_ERR_DEVICE;
        }
        owned_host.push_back(*ptr);
        return FDM_OK;
    }
    fdm_status alloc(void** ptr, size_t bytes) {
        *ptr = nullptr;
        if (injected_alloc_failure()) return FDM_ERR_OOM;
        cudaError_t e = cudaMalloc(ptr, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            *ptr = nullptr;
            return e == cudaErrorMemoryAllocation ? FDM_ERR_OOM : FDM_ERR_DEVICE;
        }
        owned.push_back(*ptr);
        return FDM_OK;
    }
    void release(void* q) {
        for (size_t i = 0; i < owned.size(); ++i)
            if (owned[i] == q) {
                cudaFree(q);
                owned.erase(owned.begin() + (long)i);
                return;
            }
    }
    void free_all() {
        for (void* q : owned) cudaFree(q);
        owned.clear();
        for (void* q : owned_host) cudaFreeHost(q);
        owned_host.clear();
    }
};

// Allocates and initialises the buffers of a group of `count` instances with parameters p
// (nz resolved): state, spectra, the layer Green kernel K (Sec. 3.1.2/3.2.1) and twiddles.
// with_spec2: second spectrum for field readouts (single instance).
template <typename T>
fdm_status build_group(Dev& d, Arena& A, const fdm_params& p, int count, int gated, bool with_spec2, cudaStream_t s);

// Uploads a host FP64 field into a device buffer of precision `prec` (FDM_FP64, FDM_MIXED,
// FDM_DF64), minus offset / downloads it, adding offset back.
fdm_status upload_field(void* dst, const double* src, size_t n, int prec, double offset, cudaStream_t s);

// Heterogeneous antiplane static problem (fdm_hetero.cu): device fields of type T, n each:
// the shear modulus, the iterate g (two components) and two work fields; gam: the Green
// operator's ratios on the quarter spectrum, 3 (n1/2+1)(n2/2+1) values (FP32 for FP32 fields,
// FP64 otherwise).
struct HeteroBuffers {
    void *mu, *g1, *g2, *t1, *t2, *gam;
};
// Runs the fixed-point iteration for the current state of the single-instance group d and
// writes sigma13 to d.tau and sigma23 to hb.t2.  stress_control: load = sigma_bar13, else
// load = eps_bar13.  tol = 0 runs exactly max_iter iterations.
template <typename T>
fdm_status hetero_solve(const Dev& d, const HeteroBuffers& hb, double mu0, bool stress_control, double load,
                        double tol, int max_iter, cudaStream_t s, int* iterations, double* residual);
// Heterogeneous static problem for a plastic layer thinner than the cell (FP64 group d, the
// current state): modulus field f_dev (device, n1 n2) uniform through the depth, reference
// factor f0; bufs: three device arrays of 12 (nz/2 + 1) n1 n2 doubles; partials: nblk x 2
// doubles.  Writes the layer average of sigma13 to tau_out (device, n1 n2) and sigma13 on the
// planes planes_dev[nplanes] to planes_out (device, nplanes n1 n2).
fdm_status hetero_layer_solve(const Dev& d, const double* f_dev, double f0, bool stress_control, double load,
                              double tol, int max_iter, const int* planes_dev, int nplanes, double* tau_out,
                              double* planes_out, void* const bufs[3], double* partials, int nblk, cudaStream_t s,
                              int* iterations, double* residual);
fdm_status download_field(double* dst, const void* src, size_t n, int prec, double offset, cudaStream_t s);
// U13 of instance `inst` in state buffer b, from / to host doubles (minus / plus `offset`);
// FDM_MIXED stores FP32 pairs: hi = fl(v), lo = fl(v - hi)
fdm_status upload_state(const Dev& d, int prec, int b, int inst, const double* src, double offset, cudaStream_t s);
fdm_status download_state(double* dst, const Dev& d, int prec, int b, int inst, double offset, cudaStream_t s);

// A step of every group as CUDA graphs (1 and kGraphSteps steps), replayed on a stream.
// Whole steps recorded as CUDA graphs.  With several groups each group's kernels form their
// own branch of the graph (captured on a side stream forked from and joined back to the
// capture stream), so independent groups run concurrently and fill the GPU together.
struct StepGraphs {
    cudaGraphExec_t one = nullptr, many = nullptr;
    cudaStream_t capture = nullptr;
    std::vector<cudaStream_t> side;   // one per group (several groups only)
    std::vector<cudaEvent_t> join;    // one per group, plus the fork event at the end
    static constexpr int kGraphSteps = 8;
    void destroy() {
        if (one) cudaGraphExecDestroy(one);
        if (many) cudaGraphExecDestroy(many);
        if (capture) cudaStreamDestroy(capture);
        for (cudaStream_t x : side) cudaStreamDestroy(x);
        for (cudaEvent_t x : join) cudaEventDestroy(x);
        one = many = nullptr;
        capture = nullptr;
        side.clear();
        join.clear();
    }
};

fdm_status build_step_graphs(StepGraphs& g, const std::vector<Dev*>& groups, const std::vector<int>& prec);
// scalars and FP64 Nye sums of instance `inst` of a group (synchronises `stream`)
fdm_status instance_info(const Dev& d, int inst, int prec, cudaStream_t stream, fdm_step_info* info);
fdm_status replay_steps(StepGraphs& g, int nsteps, cudaStream_t s);

}  // namespace fdm
