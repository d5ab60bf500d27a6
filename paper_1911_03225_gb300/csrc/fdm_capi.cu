// fdm_capi.cu -- C ABI (include/fdm.h) of a single FDM instance over the CUDA kernels:
// handle lifetime, device memory, host<->device copies, step sequencing (CUDA graphs) and
// status reporting.  Shared group/graph helpers are defined here too.
#include <cmath>
#include <cstdio>
#include <type_traits>
#include <cstring>
#include <new>
#include <vector>

#include "fdm_device.cuh"
#include "fdm_host.h"

namespace fdm {

const double kPi = 3.14159265358979323846;

// twiddle tables exp(-2 pi i m / n) and the pass tables of an L-point transform, built on
// the device by the one routine every path uses (launch_twiddle_tables)
template <typename T>
static fdm_status upload_twiddles(void* dst, int n, cudaStream_t s) {
    launch_twiddle_tables<T>(dst, n, nullptr, 0, s);
    FDM_CK(cudaGetLastError());
    return FDM_OK;
}

template <typename T>
static fdm_status upload_pass_twiddles(void* dst, int L, cudaStream_t s) {
    launch_twiddle_tables<T>(nullptr, 0, dst, L, s);
    FDM_CK(cudaGetLastError());
    return FDM_OK;
}

template <typename T>
fdm_status build_group(Dev& d, Arena& A, const fdm_params& p, int count, int gated, bool with_spec2,
                       cudaStream_t s) {
    d = Dev{};
    d.p = p;
    d.count = count;
    d.gated = gated;
    const size_t n = (size_t)p.n1 * p.n2;
    d.geom = geometry<T>(p.n1, p.n2);
    if (d.geom.row_smem > 200 * 1024 || d.geom.col_smem > 200 * 1024) return FDM_ERR_INVALID_ARG;
    FDM_CK(configure_kernels<T>());
    fdm_status st;
    const size_t cn = (size_t)count * n;
    if ((st = A.alloc(&d.phi[0], cn * sizeof(T)))) return st;
    if ((st = A.alloc(&d.phi[1], cn * sizeof(T)))) return st;
    if (std::is_same<T, float>::value) {   // FP32 pairs: low words of the state
        if ((st = A.alloc(&d.phi_lo[0], cn * sizeof(T)))) return st;
        if ((st = A.alloc(&d.phi_lo[1], cn * sizeof(T)))) return st;
        FDM_CK(cudaMemsetAsync(d.phi_lo[0], 0, cn * sizeof(T), s));
        FDM_CK(cudaMemsetAsync(d.phi_lo[1], 0, cn * sizeof(T), s));
    }
    if ((st = A.alloc(&d.tau, cn * sizeof(T)))) return st;
    if ((st = A.alloc(&d.spec, cn * sizeof(T)))) return st;   // n1/2 * n2 complex per instance
    if (with_spec2 && (st = A.alloc(&d.spec2, n * sizeof(T)))) return st;
    const size_t nk = (size_t)(p.n1 / 2 + 1) * (p.n2 / 2 + 1);
    if ((st = A.alloc(&d.Kh, nk * sizeof(T)))) return st;
    if ((st = A.alloc(&d.tw1, (size_t)p.n1 * 2 * sizeof(T)))) return st;
    if ((st = A.alloc(&d.tw2, (size_t)p.n2 * 2 * sizeof(T)))) return st;
    if ((st = A.alloc(&d.pt1, (size_t)(pass_table_len(p.n1 / 2) + 1) * 2 * sizeof(T)))) return st;
    if ((st = A.alloc(&d.pt2, (size_t)(pass_table_len(p.n2) + 1) * 2 * sizeof(T)))) return st;
    if ((st = A.alloc((void**)&d.row_partials, (size_t)count * p.n2 * sizeof(double)))) return st;
    d.red_blocks = red_blocks_for(n);
    if ((st = A.alloc((void**)&d.red, (size_t)6 * d.red_blocks * sizeof(double)))) return st;
    if ((st = A.alloc_host((void**)&d.red_host, kInfoScalarBytes + (size_t)6 * d.red_blocks * sizeof(double))))
        return st;
    if ((st = A.alloc((void**)&d.sc, (size_t)count * sizeof(fdm_dev_scalars)))) return st;
    FDM_CK(cudaMemsetAsync(d.sc, 0, (size_t)count * sizeof(fdm_dev_scalars), s));
    FDM_CK(cudaMemsetAsync(d.phi[0], 0, cn * sizeof(T), s));
    if ((st = upload_twiddles<T>(d.tw1, p.n1, s))) return st;
    if ((st = upload_twiddles<T>(d.tw2, p.n2, s))) return st;
    if ((st = upload_pass_twiddles<T>(d.pt1, p.n1 / 2, s))) return st;
    if ((st = upload_pass_twiddles<T>(d.pt2, p.n2, s))) return st;
    // layer weights |chi-hat(k3)|^2, k3 in [0, nz/2] (Sec. 3.2.1 layer of nh voxels)
    void* dw3 = nullptr;
    void* dK64 = nullptr;
    if ((st = A.alloc(&dw3, ((size_t)p.nz / 2 + 1) * sizeof(double)))) return st;
    if ((st = A.alloc(&dK64, nk * sizeof(double)))) return st;
    launch_layer_weights((double*)dw3, p.nz, p.nh, s);
    const double mu = p.E / (2.0 * (1.0 + p.nu));
    launch_kernel_table((double*)dK64, p.n1, p.n2, p.nz, p.nh, mu, p.nu, (const double*)dw3, s);
    FDM_CK(cudaGetLastError());
    launch_convert<T>((const double*)dK64, (T*)d.Kh, nk, 0.0, s);
    FDM_CK(cudaGetLastError());
    FDM_CK(cudaStreamSynchronize(s));
    A.release(dw3);
    A.release(dK64);
    if (p.autotune) {
        // times the candidate launch shapes on this group's buffers, then clears them again
        FDM_CK(autotune_group<T>(d, s));
        FDM_CK(cudaMemsetAsync(d.sc, 0, (size_t)count * sizeof(fdm_dev_scalars), s));
        FDM_CK(cudaMemsetAsync(d.phi[0], 0, cn * sizeof(T), s));
        for (void* lo : d.phi_lo)
            if (lo) FDM_CK(cudaMemsetAsync(lo, 0, cn * sizeof(T), s));
        FDM_CK(cudaStreamSynchronize(s));
    }
    return FDM_OK;
}

template fdm_status build_group<double>(Dev&, Arena&, const fdm_params&, int, int, bool, cudaStream_t);
template fdm_status build_group<float>(Dev&, Arena&, const fdm_params&, int, int, bool, cudaStream_t);
template fdm_status build_group<df>(Dev&, Arena&, const fdm_params&, int, int, bool, cudaStream_t);

fdm_status upload_field(void* dst, const double* src, size_t n, int prec, double offset, cudaStream_t s) {
    if (prec == FDM_FP64 && offset == 0.0) {
        FDM_CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, s));
        FDM_CK(cudaStreamSynchronize(s));
        return FDM_OK;
    }
    if (prec == FDM_MIXED) {
        std::vector<float> t(n);
        for (size_t i = 0; i < n; ++i) t[i] = (float)(src[i] - offset);
        FDM_CK(cudaMemcpyAsync(dst, t.data(), n * sizeof(float), cudaMemcpyHostToDevice, s));
        FDM_CK(cudaStreamSynchronize(s));
        return FDM_OK;
    }
    if (prec == FDM_DF64) {
        std::vector<df> t(n);
        for (size_t i = 0; i < n; ++i) t[i] = df(src[i] - offset);
        FDM_CK(cudaMemcpyAsync(dst, t.data(), n * sizeof(df), cudaMemcpyHostToDevice, s));
        FDM_CK(cudaStreamSynchronize(s));
        return FDM_OK;
    }
    std::vector<double> t(n);
    for (size_t i = 0; i < n; ++i) t[i] = src[i] - offset;
    FDM_CK(cudaMemcpyAsync(dst, t.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
    FDM_CK(cudaStreamSynchronize(s));
    return FDM_OK;
}

fdm_status download_field(double* dst, const void* src, size_t n, int prec, double offset, cudaStream_t s) {
    if (prec == FDM_MIXED) {
        std::vector<float> t(n);
        FDM_CK(cudaMemcpyAsync(t.data(), src, n * sizeof(float), cudaMemcpyDeviceToHost, s));
        FDM_CK(cudaStreamSynchronize(s));
        for (size_t i = 0; i < n; ++i) dst[i] = (double)t[i] + offset;
        return FDM_OK;
    }
    if (prec == FDM_DF64) {
        std::vector<df> t(n);
        FDM_CK(cudaMemcpyAsync(t.data(), src, n * sizeof(df), cudaMemcpyDeviceToHost, s));
        FDM_CK(cudaStreamSynchronize(s));
        for (size_t i = 0; i < n; ++i) dst[i] = (double)t[i] + offset;
        return FDM_OK;
    }
    FDM_CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    FDM_CK(cudaStreamSynchronize(s));
    if (offset != 0.0)
        for (size_t i = 0; i < n; ++i) dst[i] += offset;
    return FDM_OK;
}

fdm_status upload_state(const Dev& d, int prec, int b, int inst, const double* src, double offset, cudaStream_t s) {
    const size_t n = (size_t)d.p.n1 * d.p.n2;
    if (prec != FDM_MIXED)
        return upload_field((char*)d.phi[b] + (size_t)inst * n * elt_size(&d.p), src, n, prec, offset, s);
    std::vector<float> hi(n), lo(n);
    for (size_t i = 0; i < n; ++i) {
        const double v = src[i] - offset;
        hi[i] = (float)v;
        lo[i] = (float)(v - (double)hi[i]);
    }
    FDM_CK(cudaMemcpyAsync((float*)d.phi[b] + inst * n, hi.data(), n * sizeof(float), cudaMemcpyHostToDevice, s));
    FDM_CK(cudaMemcpyAsync((float*)d.phi_lo[b] + inst * n, lo.data(), n * sizeof(float), cudaMemcpyHostToDevice, s));
    FDM_CK(cudaStreamSynchronize(s));
    return FDM_OK;
}

fdm_status download_state(double* dst, const Dev& d, int prec, int b, int inst, double offset, cudaStream_t s) {
    const size_t n = (size_t)d.p.n1 * d.p.n2;
    if (prec != FDM_MIXED)
        return download_field(dst, (const char*)d.phi[b] + (size_t)inst * n * elt_size(&d.p), n, prec, offset, s);
    std::vector<float> hi(n), lo(n);
    FDM_CK(cudaMemcpyAsync(hi.data(), (const float*)d.phi[b] + inst * n, n * sizeof(float), cudaMemcpyDeviceToHost, s));
    FDM_CK(cudaMemcpyAsync(lo.data(), (const float*)d.phi_lo[b] + inst * n, n * sizeof(float), cudaMemcpyDeviceToHost, s));
    FDM_CK(cudaStreamSynchronize(s));
    for (size_t i = 0; i < n; ++i) dst[i] = ((double)hi[i] + (double)lo[i]) + offset;
    return FDM_OK;
}

static fdm_status capture_steps(cudaGraphExec_t* out, const StepGraphs& sg, int nsteps,
                                const std::vector<Dev*>& groups, const std::vector<int>& prec) {
    cudaGraph_t graph = nullptr;
    cudaStream_t cap = sg.capture;
    FDM_CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    if (groups.size() == 1) {
        for (int k = 0; k < nsteps; ++k) FDM_DISPATCH(prec[0], launch_step<T>(*groups[0], cap));
    } else {
        // fork: every group's steps on its own stream; join them all at the end
        cudaEvent_t fork = sg.join.back();
        cudaError_t r = cudaEventRecord(fork, cap);
        for (size_t g = 0; g < groups.size() && r == cudaSuccess; ++g) {
            r = cudaStreamWaitEvent(sg.side[g], fork, 0);
            for (int k = 0; k < nsteps && r == cudaSuccess; ++k) FDM_DISPATCH(prec[g], launch_step<T>(*groups[g], sg.side[g]));
            if (r == cudaSuccess) r = cudaEventRecord(sg.join[g], sg.side[g]);
            if (r == cudaSuccess) r = cudaStreamWaitEvent(cap, sg.join[g], 0);
        }
        if (r != cudaSuccess) {
            cudaStreamEndCapture(cap, &graph);
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return FDM_ERR_DEVICE;
        }
    }
    cudaError_t e = cudaStreamEndCapture(cap, &graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FDM_ERR_DEVICE;
    }
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FDM_ERR_DEVICE;
    }
    return FDM_OK;
}

fdm_status build_step_graphs(StepGraphs& g, const std::vector<Dev*>& groups, const std::vector<int>& prec) {
    if (g.one) return FDM_OK;
    if (!g.capture) FDM_CK(cudaStreamCreateWithFlags(&g.capture, cudaStreamNonBlocking));
    if (groups.size() > 1 && g.side.empty()) {
        for (size_t i = 0; i < groups.size(); ++i) {
            cudaStream_t x = nullptr;
            FDM_CK(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
            g.side.push_back(x);
        }
        for (size_t i = 0; i <= groups.size(); ++i) {
            cudaEvent_t x = nullptr;
            FDM_CK(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
            g.join.push_back(x);
        }
    }
    fdm_status st = capture_steps(&g.one, g, 1, groups, prec);
    if (st) return st;
    return capture_steps(&g.many, g, StepGraphs::kGraphSteps, groups, prec);
}

fdm_status replay_steps(StepGraphs& g, int nsteps, cudaStream_t s) {
    while (nsteps >= StepGraphs::kGraphSteps) {
        FDM_CK(cudaGraphLaunch(g.many, s));
        nsteps -= StepGraphs::kGraphSteps;
    }
    for (; nsteps > 0; --nsteps) FDM_CK(cudaGraphLaunch(g.one, s));
    return FDM_OK;
}

// FP64 sums over the staggered Nye components of one instance's current state (info)
int g_fail_alloc_countdown = -1;

fdm_status instance_info(const Dev& d, int inst, int prec, cudaStream_t stream, fdm_step_info* info) {
    // the sums read the current buffer on the device: one round trip for scalars and sums
    FDM_DISPATCH(prec, launch_alpha_sums<T>(d, inst, d.red, d.red_blocks, stream));
    FDM_CK(cudaGetLastError());
    fdm_dev_scalars* hs = (fdm_dev_scalars*)d.red_host;
    double* part = (double*)((char*)d.red_host + kInfoScalarBytes);
    FDM_CK(cudaMemcpyAsync(hs, d.sc + inst, sizeof(*hs), cudaMemcpyDeviceToHost, stream));
    FDM_CK(cudaMemcpyAsync(part, d.red, (size_t)6 * d.red_blocks * sizeof(double), cudaMemcpyDeviceToHost, stream));
    FDM_CK(cudaStreamSynchronize(stream));
    const fdm_dev_scalars s = *hs;
    const size_t n = (size_t)d.p.n1 * d.p.n2;
    double sums[6];
    std::vector<double> col(d.red_blocks);
    for (int q = 0; q < 6; ++q) {
        for (int b = 0; b < d.red_blocks; ++b) col[b] = part[6 * b + q];
        sums[q] = ksum(col.data(), col.size());
    }
    // sums of the differences d12 = dx alpha12 and d11 = -dx alpha11 (Sec. 3.2.1)
    const double idx = 1.0 / d.p.dx;
    std::memset(info, 0, sizeof(*info));
    info->step = s.step;
    info->t = s.t;
    info->dt = s.dt;
    info->max_abs_v0 = s.max_abs_v0;
    info->mean_up13 = s.phi_ref + sums[5] / (double)n;
    host_loading(d.p, s.step, s.t, info->mean_up13, &info->eps_bar13, &info->sigma_bar13);
    info->sum_a12_pos = 0.5 * (sums[0] + sums[1]) * idx;
    info->sum_a12_neg = 0.5 * (sums[1] - sums[0]) * idx;
    info->sum_a11_pos = 0.5 * (sums[2] - sums[3]) * idx;
    info->sum_a11_neg = -0.5 * (sums[2] + sums[3]) * idx;
    info->sum_abs_alpha = sums[4] * idx;
    info->status = s.status;
    return FDM_OK;
}

}  // namespace fdm

using namespace fdm;

struct fdm_handle {
    Dev d;
    Arena arena;
    StepGraphs graphs;
    cudaStream_t stream;
    int next_phase;          // next kernel of a partially enqueued step (0: none pending)
    bool has_state;
    int prec;                // FDM_FP64, FDM_MIXED or FDM_DF64
    size_t n;                // n1 * n2
    void* rd[4];             // readout buffers (type T, n each), allocated on first use
    void* mfac_buf;          // mobility factor (type T, n), allocated on first use
    void* plane_buf[5];      // stress planes: FP64 table, table in T, k3 weights, output in T, scalars
    HeteroBuffers hetero;    // heterogeneous static problem, allocated on first use
    bool hetero_on;          // steps and static solves use the shear-modulus field in hetero.mu
    double hetero_mu0, hetero_tol;
    int hetero_max_iter;
    Dev rd64;                // mixed precision: FP64 spectra and tables for the Nye readout
    void* rd64_buf[3];       //   U13 and the two Nye components in FP64 (n each)
};

namespace {

fdm_status reset_scalars(fdm_handle* h, double mean) {
    fdm_dev_scalars s;
    std::memset(&s, 0, sizeof(s));
    s.phi_ref = h->d.phi_ref_host;
    s.mean_up13 = mean;
    s.cur = 0;
    s.steps_left = -1;
    host_loading(h->d.p, 0, 0.0, mean, &s.eps_bar13, &s.sigma_bar13);
    FDM_CK(cudaMemcpyAsync(h->d.sc, &s, sizeof(s), cudaMemcpyHostToDevice, h->stream));
    FDM_CK(cudaStreamSynchronize(h->stream));
    h->next_phase = 0;
    h->has_state = true;
    return FDM_OK;
}

fdm_status read_scalars(fdm_handle* h, fdm_dev_scalars* s) {
    FDM_CK(cudaMemcpyAsync(s, h->d.sc, sizeof(*s), cudaMemcpyDeviceToHost, h->stream));
    FDM_CK(cudaStreamSynchronize(h->stream));
    return FDM_OK;
}

template <typename T>
fdm_status ensure_readout(fdm_handle* h) {
    for (int i = 0; i < 4; ++i)
        if (!h->rd[i]) {
            fdm_status st = h->arena.alloc(&h->rd[i], h->n * sizeof(T));
            if (st) return st;
        }
    return FDM_OK;
}

// The mixed path reads its Nye field out in FP64: the state's word pairs convert exactly,
// so the readout adds no FP32 transform rounding to a field whose norm may be a small
// fraction of U13's.  Spectra and tables are allocated on first use.
fdm_status ensure_readout64(fdm_handle* h) {
    Dev& r = h->rd64;
    if (r.spec) return FDM_OK;
    fdm_status st;
    const fdm_params& p = h->d.p;
    r = Dev{};
    r.p = p;
    r.p.precision = FDM_FP64;
    r.count = 1;
    FDM_CK(configure_kernels<double>());
    r.geom = geometry<double>(p.n1, p.n2);
    const size_t n = h->n;
    if ((st = h->arena.alloc(&r.spec, n * sizeof(double)))) return st;
    if ((st = h->arena.alloc(&r.spec2, n * sizeof(double)))) return st;
    if ((st = h->arena.alloc(&r.tw1, (size_t)p.n1 * 2 * sizeof(double)))) return st;
    if ((st = h->arena.alloc(&r.tw2, (size_t)p.n2 * 2 * sizeof(double)))) return st;
    if ((st = h->arena.alloc(&r.pt1, (size_t)(pass_table_len(p.n1 / 2) + 1) * 2 * sizeof(double)))) return st;
    if ((st = h->arena.alloc(&r.pt2, (size_t)(pass_table_len(p.n2) + 1) * 2 * sizeof(double)))) return st;
    if ((st = upload_twiddles<double>(r.tw1, p.n1, h->stream))) return st;
    if ((st = upload_twiddles<double>(r.tw2, p.n2, h->stream))) return st;
    if ((st = upload_pass_twiddles<double>(r.pt1, p.n1 / 2, h->stream))) return st;
    if ((st = upload_pass_twiddles<double>(r.pt2, p.n2, h->stream))) return st;
    for (int i = 0; i < 3; ++i)
        if ((st = h->arena.alloc(&h->rd64_buf[i], n * sizeof(double)))) return st;
    return FDM_OK;
}

template <typename T>
fdm_status read_fields_impl(fdm_handle* h, uint32_t mask, double* up13, double* a11, double* a12, double* tau,
                            double* v1, double* v2) {
    Dev& d = h->d;
    fdm_dev_scalars sc;
    fdm_status st;
    if ((st = read_scalars(h, &sc))) return st;
    const T* phi = (const T*)d.phi[sc.cur];
    const int mx = h->prec;
    if (mask & FDM_FIELD_UP13)
        if ((st = download_state(up13, d, mx, sc.cur, 0, d.phi_ref_host, h->stream))) return st;
    if (mask & FDM_FIELD_TAU13)
        if ((st = download_field(tau, d.tau, h->n, mx, 0.0, h->stream))) return st;
    const bool nye64 = mx == FDM_MIXED && (mask & (FDM_FIELD_ALPHA11 | FDM_FIELD_ALPHA12));
    if (nye64) {
        if ((st = ensure_readout64(h))) return st;
        double* u64 = (double*)h->rd64_buf[0];
        launch_pair_to_double((const float*)d.phi[sc.cur], (const float*)d.phi_lo[sc.cur], u64, h->n, h->stream);
        launch_alpha<double>(h->rd64, u64, (double*)h->rd64_buf[1], (double*)h->rd64_buf[2], h->stream);
        FDM_CK(cudaGetLastError());
        if (mask & FDM_FIELD_ALPHA11)
            if ((st = download_field(a11, h->rd64_buf[1], h->n, FDM_FP64, 0.0, h->stream))) return st;
        if (mask & FDM_FIELD_ALPHA12)
            if ((st = download_field(a12, h->rd64_buf[2], h->n, FDM_FP64, 0.0, h->stream))) return st;
    }
    if ((mask & (FDM_FIELD_V1 | FDM_FIELD_V2)) || (!nye64 && (mask & (FDM_FIELD_ALPHA11 | FDM_FIELD_ALPHA12)))) {
        if ((st = ensure_readout<T>(h))) return st;
        launch_alpha<T>(d, phi, (T*)h->rd[0], (T*)h->rd[1], h->stream);
        FDM_CK(cudaGetLastError());
        if ((mask & FDM_FIELD_ALPHA11) && !nye64)
            if ((st = download_field(a11, h->rd[0], h->n, mx, 0.0, h->stream))) return st;
        if ((mask & FDM_FIELD_ALPHA12) && !nye64)
            if ((st = download_field(a12, h->rd[1], h->n, mx, 0.0, h->stream))) return st;
        if (mask & (FDM_FIELD_V1 | FDM_FIELD_V2)) {
            launch_velocity<T>(d, (const T*)h->rd[0], (const T*)h->rd[1], (const T*)d.tau, phi, (T*)h->rd[2],
                               (T*)h->rd[3], h->stream);
            FDM_CK(cudaGetLastError());
            if (mask & FDM_FIELD_V1)
                if ((st = download_field(v1, h->rd[2], h->n, mx, 0.0, h->stream))) return st;
            if (mask & FDM_FIELD_V2)
                if ((st = download_field(v2, h->rd[3], h->n, mx, 0.0, h->stream))) return st;
        }
    }
    return FDM_OK;
}

}  // namespace

extern "C" {

void fdm_default_params(fdm_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->nz = 0;
    p->nh = 4;
    p->dx = 1.0;
    p->E = 1.0;
    p->nu = 0.3;
    p->velocity_mode = FDM_V_PRESCRIBED;
    p->v0 = 1.0;
    p->mobility = 1.0;
    p->tau_y = 0.0;
    p->beta = 1.0;
    p->autotune = 1;
    p->theta = 1.0;
    p->cfl = 0.5;
    p->dt_max = 0.0;
    p->loading_mode = FDM_LOAD_STRESS;
    p->time_level = FDM_T_MIDPOINT;
    p->precision = FDM_FP64;
}

size_t fdm_device_bytes(const fdm_params* p) {
    if (!params_valid(p)) return 0;
    size_t n = (size_t)p->n1 * p->n2, e = elt_size(p);
    size_t nk = (size_t)(p->n1 / 2 + 1) * (p->n2 / 2 + 1);
    const size_t lo = p->precision == FDM_MIXED ? 2 * n * sizeof(float) : 0;   // low words of the state
    return 5 * n * e + lo + nk * e + (size_t)(p->n1 + p->n2) * 4 * e + (size_t)p->n2 * sizeof(double) + 64 * 1024;
}

fdm_status fdm_create(const fdm_params* p, void* stream, fdm_handle** out) {
    if (!out) return FDM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!params_valid(p)) return FDM_ERR_INVALID_ARG;
    fdm_handle* h = new (std::nothrow) fdm_handle();
    if (!h) return FDM_ERR_OOM;
    fdm_params q = *p;
    if (q.nz == 0) q.nz = p->n1;
    h->stream = (cudaStream_t)stream;
    h->next_phase = 0;
    h->has_state = false;
    h->prec = p->precision;
    h->n = (size_t)p->n1 * p->n2;
    fdm_status st = FDM_OK;
    FDM_DISPATCH(h->prec, st = build_group<T>(h->d, h->arena, q, 1, 0, true, h->stream));
    if (st != FDM_OK) {
        fdm_destroy(h);
        return st;
    }
    h->d.phi_ref_host = 0.0;
    *out = h;
    return FDM_OK;
}

// FP64 state: the field goes to the device as it is (staged in the stress buffer, which the
// next static solve overwrites) and its mean comes from a device reduction, so that a large
// restart costs one copy rather than a host pass; the state is replaced only if the sum is
// finite.
static fdm_status set_state_fp64(fdm_handle* h, const double* up13) {
    Dev& d = h->d;
    const size_t n = h->n;
    FDM_CK(cudaStreamSynchronize(h->stream));
    FDM_CK(cudaMemcpyAsync(d.tau, up13, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    Dev r = d;
    r.phi[0] = r.phi[1] = d.tau;
    r.phi_lo[0] = r.phi_lo[1] = nullptr;
    r.sc = nullptr;
    launch_alpha_sums<double>(r, 0, d.red, d.red_blocks, h->stream);
    FDM_CK(cudaGetLastError());
    double* part = (double*)((char*)d.red_host + kInfoScalarBytes);
    FDM_CK(cudaMemcpyAsync(part, d.red, (size_t)6 * d.red_blocks * sizeof(double), cudaMemcpyDeviceToHost,
                           h->stream));
    FDM_CK(cudaStreamSynchronize(h->stream));
    std::vector<double> col(d.red_blocks);
    for (int b = 0; b < d.red_blocks; ++b) col[b] = part[6 * b + 5];
    const double mean = ksum(col.data(), col.size()) / (double)n;
    if (!std::isfinite(mean)) return FDM_ERR_INVALID_ARG;
    FDM_CK(cudaMemcpyAsync(d.phi[0], d.tau, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    d.phi_ref_host = 0.0;
    return reset_scalars(h, mean);
}

fdm_status fdm_set_plastic_distortion(fdm_handle* h, const double* up13) {
    if (!h || !up13) return FDM_ERR_INVALID_ARG;
    if (h->prec == FDM_FP64) return set_state_fp64(h, up13);
    double mean = ksum(up13, h->n) / (double)h->n;
    if (!std::isfinite(mean)) return FDM_ERR_INVALID_ARG;
    FDM_CK(cudaStreamSynchronize(h->stream));
    // FP32 and double-word storage hold U13 minus its mean (the scheme is offset equivariant)
    h->d.phi_ref_host = h->prec != FDM_FP64 ? mean : 0.0;
    fdm_status st = upload_state(h->d, h->prec, 0, 0, up13, h->d.phi_ref_host, h->stream);
    if (st) return st;
    return reset_scalars(h, mean);
}

fdm_status fdm_set_density(fdm_handle* h, const double* a11, const double* a12, double mean_up13,
                           double* div_residual) {
    if (!h || !a11 || !a12 || !std::isfinite(mean_up13)) return FDM_ERR_INVALID_ARG;
    const size_t n = h->n;
    double m11 = ksum(a11, n) / (double)n, m12 = ksum(a12, n) / (double)n, amax = 0.0;
    for (size_t i = 0; i < n; ++i) {
        if (!std::isfinite(a11[i]) || !std::isfinite(a12[i])) return FDM_ERR_INVALID_ARG;
        amax = std::fmax(amax, std::fmax(std::fabs(a11[i]), std::fabs(a12[i])));
    }
    if (std::fabs(m11) > 1e-9 * amax || std::fabs(m12) > 1e-9 * amax) return FDM_ERR_NET_BURGERS;
    FDM_CK(cudaStreamSynchronize(h->stream));
    Dev& d = h->d;
    fdm_status st;
    // stage alpha in the two state buffers (the old state is being replaced)
    if ((st = upload_field(d.phi[0], a11, n, h->prec, 0.0, h->stream))) return st;
    if ((st = upload_field(d.phi[1], a12, n, h->prec, 0.0, h->stream))) return st;
    double phi_ref = h->prec != FDM_FP64 ? mean_up13 : 0.0;
    const int nblk = d.red_blocks;
    FDM_DISPATCH(h->prec, launch_curl_inverse<T>(d, (const T*)d.phi[0], (const T*)d.phi[1], (T*)d.phi[0], mean_up13,
                                                 phi_ref, d.red, nblk, h->stream));
    FDM_CK(cudaGetLastError());
    std::vector<double> part((size_t)2 * nblk);
    FDM_CK(cudaMemcpyAsync(part.data(), d.red, part.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    FDM_CK(cudaStreamSynchronize(h->stream));
    double num = 0.0, den = 0.0;
    for (int b = 0; b < nblk; ++b) { num += part[2 * b]; den += part[2 * b + 1]; }
    double res = den > 0.0 ? std::sqrt(num / den) : 0.0;
    if (div_residual) *div_residual = res;
    d.phi_ref_host = phi_ref;
    if (d.phi_lo[0]) FDM_CK(cudaMemsetAsync(d.phi_lo[0], 0, n * sizeof(float), h->stream));
    if ((st = reset_scalars(h, mean_up13))) return st;
    return res > 1e-6 ? FDM_WARN_NOT_DIV_FREE : FDM_OK;
}

fdm_status fdm_set_clock(fdm_handle* h, int64_t step, double t) {
    if (!h || step < 0 || !std::isfinite(t)) return FDM_ERR_INVALID_ARG;
    if (!h->has_state) return FDM_ERR_STATE;
    fdm_dev_scalars s;
    fdm_status st = read_scalars(h, &s);
    if (st) return st;
    s.step = step;
    s.t = t;
    FDM_CK(cudaMemcpyAsync(h->d.sc, &s, sizeof(s), cudaMemcpyHostToDevice, h->stream));
    FDM_CK(cudaStreamSynchronize(h->stream));
    return FDM_OK;
}

// buffers of the heterogeneous static problem, allocated on first use
static fdm_status alloc_hetero(fdm_handle* h) {
    const fdm_params& p = h->d.p;
    const size_t bytes = h->n * elt_size(&p);
    const size_t tab = (size_t)3 * (p.n1 / 2 + 1) * (p.n2 / 2 + 1) * (h->prec == FDM_MIXED ? sizeof(float) : sizeof(double));
    void** bufs[6] = {&h->hetero.mu, &h->hetero.g1, &h->hetero.g2, &h->hetero.t1, &h->hetero.t2, &h->hetero.gam};
    const size_t sizes[6] = {bytes, bytes, bytes, bytes, bytes, tab};
    fdm_status st;
    for (int i = 0; i < 6; ++i)
        if (!*bufs[i] && (st = h->arena.alloc(bufs[i], sizes[i]))) return st;
    return FDM_OK;
}

// the static problem of the current step with the handle's shear-modulus field (tau13 in d.tau)
static fdm_status hetero_static(fdm_handle* h, int* iterations, double* residual) {
    const fdm_params& p = h->d.p;
    fdm_dev_scalars s;
    fdm_status st;
    if ((st = read_scalars(h, &s))) return st;
    double eps = 0.0, sig = 0.0;
    host_loading(p, s.step, s.t, s.mean_up13, &eps, &sig);
    const bool stress = p.loading_mode == FDM_LOAD_STRESS || p.loading_mode == FDM_LOAD_ZERO_MEAN_STRESS;
    FDM_DISPATCH(h->prec, st = hetero_solve<T>(h->d, h->hetero, h->hetero_mu0, stress, stress ? sig : eps,
                                               h->hetero_tol, h->hetero_max_iter, h->stream, iterations, residual));
    return st;
}

// one step with the heterogeneous static problem: the iteration, the CFL step from its
// tau13, then the transport kernel (which advances step and time and flips the buffers)
static fdm_status hetero_step(fdm_handle* h) {
    int it = 0;
    double r = 0.0;
    fdm_status st = hetero_static(h, &it, &r);
    if (st) return st;
    FDM_DISPATCH(h->prec, launch_celerity_dt<T>(h->d, h->stream); launch_phase<T>(h->d, kKernelsPerStep - 1, h->stream));
    FDM_CK(cudaGetLastError());
    return FDM_OK;
}

fdm_status fdm_set_shear_modulus_field(fdm_handle* h, const double* mu_factor, double tol, int32_t max_iter) {
    if (!h) return FDM_ERR_INVALID_ARG;
    if (!mu_factor) {
        h->hetero_on = false;
        return FDM_OK;
    }
    const fdm_params& p = h->d.p;
    if (p.nh != p.nz || !(tol >= 0.0) || !std::isfinite(tol) || max_iter < 1) return FDM_ERR_INVALID_ARG;
    const size_t n = h->n;
    const double mu = p.E / (2.0 * (1.0 + p.nu));
    std::vector<double> m(n);
    double mmin = HUGE_VAL, mmax = 0.0;
    for (size_t i = 0; i < n; ++i) {
        if (!(mu_factor[i] > 0.0) || !std::isfinite(mu_factor[i])) return FDM_ERR_INVALID_ARG;
        m[i] = mu * mu_factor[i];
        mmin = std::fmin(mmin, m[i]);
        mmax = std::fmax(mmax, m[i]);
    }
    if (h->next_phase != 0) return FDM_ERR_STATE;
    fdm_status st;
    if ((st = alloc_hetero(h))) return st;
    FDM_CK(cudaStreamSynchronize(h->stream));
    if ((st = upload_field(h->hetero.mu, m.data(), n, h->prec, 0.0, h->stream))) return st;
    h->hetero_mu0 = 0.5 * (mmin + mmax);
    h->hetero_tol = tol;
    h->hetero_max_iter = max_iter;
    h->hetero_on = true;
    return FDM_OK;
}

fdm_status fdm_static_solve(fdm_handle* h) {
    if (!h) return FDM_ERR_INVALID_ARG;
    if (!h->has_state || h->next_phase != 0) return FDM_ERR_STATE;
    if (h->hetero_on) {
        int it = 0;
        double r = 0.0;
        fdm_status st = hetero_static(h, &it, &r);
        if (st) return st;
        FDM_CK(cudaStreamSynchronize(h->stream));
        return FDM_OK;
    }
    Dev& d = h->d;
    FDM_DISPATCH(h->prec, launch_static<T>(d, h->stream));
    FDM_CK(cudaGetLastError());
    // the stencil kernel normally clears the running max; no step follows here
    FDM_CK(cudaMemsetAsync(&d.sc->vmax_bits, 0, sizeof(unsigned long long), h->stream));
    FDM_CK(cudaStreamSynchronize(h->stream));
    return FDM_OK;
}

fdm_status fdm_enqueue_steps(fdm_handle* h, int32_t nsteps) {
    if (!h || nsteps < 0) return FDM_ERR_INVALID_ARG;
    if (!h->has_state || h->next_phase != 0) return FDM_ERR_STATE;
    if (nsteps == 0) return FDM_OK;
    if (h->hetero_on) {   // the iteration decides on the host: steps run on the host's loop
        for (int32_t k = 0; k < nsteps; ++k) {
            fdm_status st = hetero_step(h);
            if (st) return st;
        }
        return FDM_OK;
    }
    std::vector<Dev*> groups{&h->d};
    std::vector<int> prec{h->prec};
    fdm_status st = build_step_graphs(h->graphs, groups, prec);
    if (st) return st;
    return replay_steps(h->graphs, nsteps, h->stream);
}

fdm_status fdm_enqueue_phase(fdm_handle* h, int32_t phase) {
    if (!h || phase < 0 || phase >= kKernelsPerStep) return FDM_ERR_INVALID_ARG;
    if (!h->has_state || phase != h->next_phase || h->hetero_on) return FDM_ERR_STATE;
    FDM_DISPATCH(h->prec, launch_phase<T>(h->d, phase, h->stream));
    FDM_CK(cudaGetLastError());
    h->next_phase = (phase + 1) % kKernelsPerStep;
    return FDM_OK;
}

fdm_status fdm_sync(fdm_handle* h) {
    if (!h) return FDM_ERR_INVALID_ARG;
    if (!h->has_state) return FDM_ERR_STATE;
    fdm_dev_scalars s;
    fdm_status st = read_scalars(h, &s);
    if (st) return st;
    return s.status ? (fdm_status)s.status : FDM_OK;
}

fdm_status fdm_step(fdm_handle* h, int32_t nsteps, fdm_step_info* info) {
    fdm_status st = fdm_enqueue_steps(h, nsteps);
    if (st) return st;
    if (info) {
        if ((st = instance_info(h->d, 0, h->prec, h->stream, info))) return st;
        return info->status ? (fdm_status)info->status : FDM_OK;
    }
    return fdm_sync(h);
}

fdm_status fdm_read_fields(fdm_handle* h, uint32_t mask, double* up13, double* a11, double* a12, double* tau,
                           double* v1, double* v2) {
    if (!h) return FDM_ERR_INVALID_ARG;
    if (mask & ~63u) return FDM_ERR_INVALID_ARG;
    if (((mask & FDM_FIELD_UP13) && !up13) || ((mask & FDM_FIELD_ALPHA11) && !a11) ||
        ((mask & FDM_FIELD_ALPHA12) && !a12) || ((mask & FDM_FIELD_TAU13) && !tau) ||
        ((mask & FDM_FIELD_V1) && !v1) || ((mask & FDM_FIELD_V2) && !v2))
        return FDM_ERR_INVALID_ARG;
    if (!h->has_state) return FDM_ERR_STATE;
    fdm_status st = FDM_OK;
    FDM_DISPATCH(h->prec, st = read_fields_impl<T>(h, mask, up13, a11, a12, tau, v1, v2));
    return st;
}

fdm_status fdm_get_info(fdm_handle* h, fdm_step_info* info) {
    if (!h || !info) return FDM_ERR_INVALID_ARG;
    if (!h->has_state) return FDM_ERR_STATE;
    return instance_info(h->d, 0, h->prec, h->stream, info);
}

int32_t fdm_kernels_per_step(const fdm_handle* h) {
    (void)h;
    return kKernelsPerStep;
}

// Stress component comp on planes of the 3-D cell.  13 keeps the layer kernel's table (cos
// weights, macroscopic stress at DC); the others take the component's table with cos or sin
// weights and the symmetric or odd, real or imaginary column multiplier.
static fdm_status read_stress_planes(fdm_handle* h, int32_t comp, int32_t nplanes, const int32_t* planes,
                                     double* out) {
    if (!h || comp < FDM_S11 || comp > FDM_S12 || nplanes < 0 || (nplanes > 0 && (!planes || !out)))
        return FDM_ERR_INVALID_ARG;
    const fdm_params& p = h->d.p;
    for (int32_t k = 0; k < nplanes; ++k)
        if (planes[k] < 0 || planes[k] >= p.nz) return FDM_ERR_INVALID_ARG;
    if (!h->has_state) return FDM_ERR_STATE;
    if (h->next_phase != 0) return FDM_ERR_STATE;
    const size_t nk = (size_t)(p.n1 / 2 + 1) * (p.n2 / 2 + 1), e = elt_size(&p);
    const size_t sizes[5] = {nk * sizeof(double), nk * e, ((size_t)p.nz / 2 + 1) * sizeof(double), h->n * e,
                             sizeof(fdm_dev_scalars)};
    fdm_status st;
    for (int i = 0; i < 5; ++i)
        if (!h->plane_buf[i] && (st = h->arena.alloc(&h->plane_buf[i], sizes[i]))) return st;
    const double mu = p.E / (2.0 * (1.0 + p.nu));
    // the symbols of 11, 22, 33 and 12 are odd in n3: their sum over k3 pairs +k3 with -k3
    // into i sin; the unpaired x3 Nyquist term is dropped
    const bool odd3 = comp != FDM_S13 && comp != FDM_S23;
    std::vector<double> w((size_t)p.nz / 2 + 1);
    std::vector<double> host((size_t)h->n);
    for (int32_t k = 0; k < nplanes; ++k) {
        // weights D(k3) cos (or sin) of 2 pi k3 (x3 - (nh - 1)/2) / nz, k3 in [0, nz/2]
        const double shift = (double)planes[k] - 0.5 * (double)(p.nh - 1);
        for (int k3 = 0; k3 <= p.nz / 2; ++k3) {
            const double D = k3 == 0 ? (double)p.nh
                                     : std::sin(kPi * (double)k3 * p.nh / p.nz) / std::sin(kPi * (double)k3 / p.nz);
            const double a = 2.0 * kPi * (double)k3 * shift / (double)p.nz;
            w[k3] = odd3 ? (2 * k3 == p.nz ? 0.0 : D * std::sin(a)) : D * std::cos(a);
        }
        FDM_CK(cudaMemcpyAsync(h->plane_buf[2], w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice,
                               h->stream));
        // the layer-average table divides by nz nh; a single plane divides by nz only
        if (comp == FDM_S13)
            launch_kernel_table((double*)h->plane_buf[0], p.n1, p.n2, p.nz, 1, mu, p.nu,
                                (const double*)h->plane_buf[2], h->stream);
        else
            launch_stress_table((double*)h->plane_buf[0], p.n1, p.n2, p.nz, comp, mu, p.nu,
                                (const double*)h->plane_buf[2], h->stream);
        FDM_CK(cudaGetLastError());
        Dev r = h->d;            // the handle's buffers with the plane's table and a copy of the scalars
        r.Kh = h->plane_buf[1];
        r.sc = (fdm_dev_scalars*)h->plane_buf[4];
        FDM_CK(cudaMemcpyAsync(r.sc, h->d.sc, sizeof(fdm_dev_scalars), cudaMemcpyDeviceToDevice, h->stream));
        if (comp == FDM_S13) {
            FDM_DISPATCH(h->prec, launch_convert<T>((const double*)h->plane_buf[0], (T*)r.Kh, nk, 0.0, h->stream);
                         launch_static_to<T>(r, (T*)h->plane_buf[3], h->stream));
        } else {
            FDM_DISPATCH(h->prec, launch_convert<T>((const double*)h->plane_buf[0], (T*)r.Kh, nk, 0.0, h->stream);
                         launch_stress_to<T>(r, comp, (T*)h->plane_buf[3], h->stream));
        }
        FDM_CK(cudaGetLastError());
        if ((st = download_field(host.data(), h->plane_buf[3], h->n, h->prec, 0.0, h->stream))) return st;
        std::memcpy(out + (size_t)k * h->n, host.data(), h->n * sizeof(double));
    }
    return FDM_OK;
}

fdm_status fdm_static_solve_heterogeneous(fdm_handle* h, const double* mu_factor, double tol, int32_t max_iter,
                                          double* sigma13, double* sigma23, int32_t* iterations, double* residual) {
    if (!h || !mu_factor || !(tol >= 0.0) || !std::isfinite(tol) || max_iter < 1) return FDM_ERR_INVALID_ARG;
    const fdm_params& p = h->d.p;
    if (p.nh != p.nz) return FDM_ERR_INVALID_ARG;
    const size_t n = h->n;
    const double mu = p.E / (2.0 * (1.0 + p.nu));
    std::vector<double> m(n);
    double mmin = HUGE_VAL, mmax = 0.0;
    for (size_t i = 0; i < n; ++i) {
        if (!(mu_factor[i] > 0.0) || !std::isfinite(mu_factor[i])) return FDM_ERR_INVALID_ARG;
        m[i] = mu * mu_factor[i];
        mmin = std::fmin(mmin, m[i]);
        mmax = std::fmax(mmax, m[i]);
    }
    if (!h->has_state || h->next_phase != 0) return FDM_ERR_STATE;
    fdm_status st;
    if ((st = alloc_hetero(h))) return st;
    if ((st = upload_field(h->hetero.mu, m.data(), n, h->prec, 0.0, h->stream))) return st;
    // the loading of the current step: sigma_bar13 (stress, zero mean stress) or eps_bar13
    fdm_dev_scalars s;
    if ((st = read_scalars(h, &s))) return st;
    double eps = 0.0, sig = 0.0;
    host_loading(p, s.step, s.t, s.mean_up13, &eps, &sig);
    const bool stress = p.loading_mode == FDM_LOAD_STRESS || p.loading_mode == FDM_LOAD_ZERO_MEAN_STRESS;
    int it = 0;
    double r = 0.0;
    FDM_DISPATCH(h->prec, st = hetero_solve<T>(h->d, h->hetero, 0.5 * (mmin + mmax), stress, stress ? sig : eps, tol,
                                               max_iter, h->stream, &it, &r));
    if (st) return st;
    if (h->hetero_on) {   // the uploaded field replaces the stepping field
        h->hetero_mu0 = 0.5 * (mmin + mmax);
        h->hetero_tol = tol;
        h->hetero_max_iter = max_iter;
    }
    if (sigma13 && (st = download_field(sigma13, h->d.tau, n, h->prec, 0.0, h->stream))) return st;
    if (sigma23 && (st = download_field(sigma23, h->hetero.t2, n, h->prec, 0.0, h->stream))) return st;
    FDM_CK(cudaStreamSynchronize(h->stream));
    if (iterations) *iterations = it;
    if (residual) *residual = r;
    return FDM_OK;
}

fdm_status fdm_static_solve_heterogeneous_layer(fdm_handle* h, const double* mu_factor, double tol, int32_t max_iter,
                                                double* tau13, int32_t nplanes, const int32_t* planes,
                                                double* sigma13_planes, int32_t* iterations, double* residual) {
    if (!h || !mu_factor || !tau13 || !(tol >= 0.0) || !std::isfinite(tol) || max_iter < 1 || nplanes < 0)
        return FDM_ERR_INVALID_ARG;
    const fdm_params& p = h->d.p;
    if (h->prec != FDM_FP64 || p.nz < 2 || (p.nz & 1)) return FDM_ERR_INVALID_ARG;
    if (nplanes > 0 && (!planes || !sigma13_planes)) return FDM_ERR_INVALID_ARG;
    for (int32_t k = 0; k < nplanes; ++k)
        if (planes[k] < 0 || planes[k] >= p.nz) return FDM_ERR_INVALID_ARG;
    const size_t n = h->n;
    double fmin = HUGE_VAL, fmax = 0.0;
    for (size_t i = 0; i < n; ++i) {
        if (!(mu_factor[i] > 0.0) || !std::isfinite(mu_factor[i])) return FDM_ERR_INVALID_ARG;
        fmin = std::fmin(fmin, mu_factor[i]);
        fmax = std::fmax(fmax, mu_factor[i]);
    }
    if (!h->has_state || h->next_phase != 0) return FDM_ERR_STATE;
    fdm_dev_scalars s;
    fdm_status st;
    if ((st = read_scalars(h, &s))) return st;
    double eps = 0.0, sig = 0.0;
    host_loading(p, s.step, s.t, s.mean_up13, &eps, &sig);
    const bool stress = p.loading_mode == FDM_LOAD_STRESS || p.loading_mode == FDM_LOAD_ZERO_MEAN_STRESS;
    // device memory of this solve only: the modulus field, three sets of 12 (nz/2 + 1) fields,
    // the outputs and the reduction partials
    const size_t fields = (size_t)12 * (p.nz / 2 + 1) * n;
    const int nblk = red_blocks_for(fields);
    void* f_dev = nullptr;
    void* bufs[3] = {nullptr, nullptr, nullptr};
    void *tau_dev = nullptr, *planes_dev = nullptr, *out_dev = nullptr, *part = nullptr;
    auto release = [&]() {
        for (void* q : {f_dev, bufs[0], bufs[1], bufs[2], tau_dev, planes_dev, out_dev, part})
            if (q) h->arena.release(q);
    };
    st = h->arena.alloc(&f_dev, n * sizeof(double));
    for (int b = 0; b < 3 && !st; ++b) st = h->arena.alloc(&bufs[b], fields * sizeof(double));
    if (!st) st = h->arena.alloc(&tau_dev, n * sizeof(double));
    if (!st) st = h->arena.alloc(&part, (size_t)2 * nblk * sizeof(double));
    if (!st && nplanes > 0) st = h->arena.alloc(&planes_dev, (size_t)nplanes * sizeof(int32_t));
    if (!st && nplanes > 0) st = h->arena.alloc(&out_dev, (size_t)nplanes * n * sizeof(double));
    if (st) {
        release();
        return st;
    }
    int it = 0;
    double r = 0.0;
    do {
        if (cudaMemcpyAsync(f_dev, mu_factor, n * sizeof(double), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
            (nplanes > 0 && cudaMemcpyAsync(planes_dev, planes, (size_t)nplanes * sizeof(int32_t),
                                            cudaMemcpyHostToDevice, h->stream) != cudaSuccess)) {
            cudaGetLastError();
            st = FDM_ERR_DEVICE;
            break;
        }
        st = hetero_layer_solve(h->d, (const double*)f_dev, 0.5 * (fmin + fmax), stress, stress ? sig : eps, tol,
                                max_iter, (const int*)planes_dev, nplanes, (double*)tau_dev, (double*)out_dev, bufs,
                                (double*)part, nblk, h->stream, &it, &r);
        if (st) break;
        if (cudaMemcpyAsync(tau13, tau_dev, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
            (nplanes > 0 && cudaMemcpyAsync(sigma13_planes, out_dev, (size_t)nplanes * n * sizeof(double),
                                            cudaMemcpyDeviceToHost, h->stream) != cudaSuccess) ||
            cudaStreamSynchronize(h->stream) != cudaSuccess) {
            cudaGetLastError();
            st = FDM_ERR_DEVICE;
        }
    } while (0);
    cudaStreamSynchronize(h->stream);
    release();
    if (st) return st;
    if (iterations) *iterations = it;
    if (residual) *residual = r;
    return FDM_OK;
}

fdm_status fdm_equilibrate(fdm_handle* h, double tol, int32_t chunk, int64_t max_steps, int64_t* taken,
                           double* change) {
    if (!h || !(tol > 0.0) || !std::isfinite(tol) || chunk < 1 || max_steps < 0) return FDM_ERR_INVALID_ARG;
    if (!h->has_state) return FDM_ERR_STATE;
    const fdm_params& p = h->d.p;
    fdm_status st = fdm_set_loading(h, FDM_LOAD_ZERO_MEAN_STRESS, p.sigma_bar13, p.eps_bar13_0, p.eps_bar13_rate);
    if (st) return st;
    const size_t n = h->n;
    const int nblk = red_blocks_for(n);
    void* prev = nullptr;
    void* part = nullptr;
    if ((st = h->arena.alloc(&prev, n * sizeof(double)))) return st;
    if ((st = h->arena.alloc(&part, (size_t)2 * nblk * sizeof(double)))) {
        h->arena.release(prev);
        return st;
    }
    int64_t done = 0;
    double rel = HUGE_VAL;
    std::vector<double> buf(2 * (size_t)nblk), col(nblk);
    FDM_DISPATCH(h->prec, launch_state_change<T>(h->d, (double*)prev, 1, (double*)part, nblk, h->stream));
    while (st == FDM_OK && done < max_steps) {
        const int32_t k = (int32_t)std::min<int64_t>(chunk, max_steps - done);
        if ((st = fdm_enqueue_steps(h, k))) break;
        FDM_DISPATCH(h->prec, launch_state_change<T>(h->d, (double*)prev, 0, (double*)part, nblk, h->stream));
        if (cudaMemcpyAsync(buf.data(), part, buf.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess) {
            cudaGetLastError();
            st = FDM_ERR_DEVICE;
            break;
        }
        if ((st = fdm_sync(h))) break;   // device-side errors of the chunk's steps
        done += k;
        double sums[2];
        for (int q = 0; q < 2; ++q) {
            for (int b = 0; b < nblk; ++b) col[b] = buf[2 * (size_t)b + q];
            sums[q] = ksum(col.data(), col.size());
        }
        rel = std::sqrt(sums[0]) / std::max(std::sqrt(sums[1]), 1e-300);
        if (!std::isfinite(rel)) {
            st = FDM_ERR_NONFINITE;
            break;
        }
        if (rel < tol) break;
    }
    cudaStreamSynchronize(h->stream);
    h->arena.release(prev);
    h->arena.release(part);
    if (taken) *taken = done;
    if (change) *change = rel;
    return st;
}

fdm_status fdm_read_stress13_planes(fdm_handle* h, int32_t nplanes, const int32_t* planes, double* out) {
    return read_stress_planes(h, FDM_S13, nplanes, planes, out);
}

fdm_status fdm_read_stress_planes(fdm_handle* h, int32_t comp, int32_t nplanes, const int32_t* planes,
                                  double* out) {
    return read_stress_planes(h, comp, nplanes, planes, out);
}

fdm_status fdm_set_loading(fdm_handle* h, int32_t mode, double sigma_bar13, double eps_bar13_0,
                           double eps_bar13_rate) {
    if (!h) return FDM_ERR_INVALID_ARG;
    fdm_params q = h->d.p;
    q.loading_mode = mode;
    q.sigma_bar13 = sigma_bar13;
    q.eps_bar13_0 = eps_bar13_0;
    q.eps_bar13_rate = eps_bar13_rate;
    if (!params_valid(&q)) return FDM_ERR_INVALID_ARG;
    if (h->next_phase != 0) return FDM_ERR_STATE;
    FDM_CK(cudaStreamSynchronize(h->stream));
    h->graphs.destroy();   // the column kernel was captured with the previous loading
    h->d.p = q;
    return FDM_OK;
}

fdm_status fdm_set_mobility_field(fdm_handle* h, const double* factor) {
    if (!h) return FDM_ERR_INVALID_ARG;
    if (h->next_phase != 0) return FDM_ERR_STATE;
    if (factor)
        for (size_t i = 0; i < h->n; ++i)
            if (!std::isfinite(factor[i]) || factor[i] < 0.0) return FDM_ERR_INVALID_ARG;
    FDM_CK(cudaStreamSynchronize(h->stream));
    h->graphs.destroy();   // the step kernels were captured with the previous field
    if (!factor) {
        h->d.mfac = nullptr;   // the buffer stays owned by the arena for later use
        return FDM_OK;
    }
    if (!h->mfac_buf) {
        fdm_status st = h->arena.alloc(&h->mfac_buf, h->n * elt_size(&h->d.p));
        if (st) return st;
    }
    fdm_status st = upload_field(h->mfac_buf, factor, h->n, h->prec, 0.0, h->stream);
    if (st) return st;
    h->d.mfac = h->mfac_buf;
    return FDM_OK;
}

fdm_status fdm_get_launch_config(const fdm_handle* h, fdm_launch_config* cfg) {
    if (!h || !cfg) return FDM_ERR_INVALID_ARG;
    FDM_DISPATCH(h->prec, launch_config<T>(h->d.geom, cfg));
    return FDM_OK;
}

int32_t fdm_launch_candidates(const fdm_params* p, fdm_launch_config* out, int32_t max) {
    if (!params_valid(p) || max < 0 || (max > 0 && !out)) return 0;
    int count = 0;
    FDM_DISPATCH(p->precision, count = launch_candidates<T>(*p, out, max));
    return count;
}

fdm_status fdm_set_launch_config(fdm_handle* h, const fdm_launch_config* cfg) {
    if (!h || !cfg) return FDM_ERR_INVALID_ARG;
    if (h->next_phase != 0) return FDM_ERR_STATE;
    bool ok = false;
    LaunchGeom g{};
    FDM_DISPATCH(h->prec, ok = geometry_from_config<T>(h->d.p, *cfg, &g));
    if (!ok) return FDM_ERR_INVALID_ARG;
    FDM_CK(cudaStreamSynchronize(h->stream));
    h->graphs.destroy();   // captured with the old shapes
    h->d.geom = g;
    return FDM_OK;
}

void fdm_debug_fail_allocation(int32_t n) { g_fail_alloc_countdown = n < 0 ? -1 : n; }

void fdm_destroy(fdm_handle* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    h->graphs.destroy();
    h->arena.free_all();
    delete h;
}

const char* fdm_status_str(fdm_status s) {
    switch (s) {
        case FDM_OK: return "ok";
        case FDM_ERR_INVALID_ARG: return "invalid argument";
        case FDM_ERR_OOM: return "device out of memory";
        case FDM_ERR_NET_BURGERS: return "Nye field has a net Burgers vector (non-zero mean)";
        case FDM_WARN_NOT_DIV_FREE: return "Nye field is not divergence-free; its divergence-free part was used";
        case FDM_ERR_NONFINITE: return "non-finite time step or field";
        case FDM_ERR_TIMEOUT: return "device-side wait timed out";
        case FDM_ERR_DEVICE: return "CUDA error";
        case FDM_ERR_STATE: return "call out of order (no state set)";
        case FDM_ERR_TOO_LARGE: return "grid exceeds the fixed scratch of the no-allocation static solve (n1, n2 <= 256, nz <= 4096)";
    }
    return "unknown status";
}

}  // extern "C"
