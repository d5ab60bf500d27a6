// fdm_capi.cu -- C ABI (include/fdm.h) over the CUDA kernels: handle lifetime, device
// memory, host<->device copies, step sequencing and status reporting.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "fdm_internal.h"

using namespace fdm;

struct fdm_handle {
    Dev d;
    cudaStream_t stream;
    int cur;                 // index of the current state buffer
    int next_phase;          // next kernel of a partially enqueued step (0: none pending)
    bool has_state;
    bool mixed;
    size_t n;                // n1 * n2
    // lazily allocated readout buffers (type T, n each)
    void* rd[4];
    std::vector<void*> owned;
};

namespace {

const double kPi = 3.14159265358979323846;

bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

bool valid(const fdm_params* p) {
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
    if (p->loading_mode < FDM_LOAD_STRESS || p->loading_mode > FDM_LOAD_ZERO_MEAN_STRESS) return false;
    if (!std::isfinite(p->sigma_bar13) || !std::isfinite(p->eps_bar13_0) || !std::isfinite(p->eps_bar13_rate))
        return false;
    if (p->time_level != FDM_T_MIDPOINT && p->time_level != FDM_T_LITERAL) return false;
    if (p->precision != FDM_FP64 && p->precision != FDM_MIXED) return false;
    return true;
}

size_t elt(const fdm_params* p) { return p->precision == FDM_MIXED ? sizeof(float) : sizeof(double); }

int red_blocks_for(size_t n) {
    size_t b = (n + 255) / 256;
    if (b > 1024) b = 1024;
    return (int)b;
}

void host_loading(const fdm_params& p, long long step, double mean, double* eps, double* sig) {
    const double mu = p.E / (2.0 * (1.0 + p.nu));
    const double frac = (double)p.nh / (double)p.nz;
    if (p.loading_mode == FDM_LOAD_STRESS) {
        *sig = p.sigma_bar13;
        *eps = (p.sigma_bar13 + mu * frac * mean) / (2.0 * mu);
    } else if (p.loading_mode == FDM_LOAD_STRAIN_RAMP) {
        *eps = p.eps_bar13_0 + p.eps_bar13_rate * (double)step;
        *sig = 2.0 * mu * (*eps) - mu * frac * mean;
    } else {
        *eps = 0.5 * frac * mean;
        *sig = 0.0;
    }
}

// Neumaier sum of host values
double ksum(const double* x, size_t n) {
    double s = 0.0, c = 0.0;
    for (size_t i = 0; i < n; ++i) {
        double t = s + x[i];
        c += (std::fabs(s) >= std::fabs(x[i])) ? (s - t) + x[i] : (x[i] - t) + s;
        s = t;
    }
    return s + c;
}

fdm_status dev_alloc(fdm_handle* h, void** ptr, size_t bytes) {
    *ptr = nullptr;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return e == cudaErrorMemoryAllocation ? FDM_ERR_OOM : FDM_ERR_DEVICE;
    }
    h->owned.push_back(*ptr);
    return FDM_OK;
}

#define CK(x)                                              \
    do {                                                   \
        cudaError_t e_ = (x);                              \
        if (e_ != cudaSuccess) {                           \
            cudaGetLastError();                            \
            return FDM_ERR_DEVICE;                         \
        }                                                  \
    } while (0)

template <typename T>
fdm_status upload_twiddles(fdm_handle* h, void* dst, int n) {
    std::vector<T> tw(2 * (size_t)n);
    for (int m = 0; m < n; ++m) {
        double a = 2.0 * kPi * (double)m / (double)n;
        tw[2 * m] = (T)std::cos(a);
        tw[2 * m + 1] = (T)(-std::sin(a));
    }
    CK(cudaMemcpyAsync(dst, tw.data(), tw.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return FDM_OK;
}

template <typename T>
fdm_status create_impl(fdm_handle* h) {
    Dev& d = h->d;
    const fdm_params& p = d.p;
    const size_t n = h->n;
    d.geom = geometry<T>(p.n1, p.n2);
    if (d.geom.row_smem > 200 * 1024 || d.geom.col_smem > 200 * 1024) return FDM_ERR_INVALID_ARG;
    CK(configure_kernels<T>());
    fdm_status st;
    if ((st = dev_alloc(h, &d.phi[0], n * sizeof(T)))) return st;
    if ((st = dev_alloc(h, &d.phi[1], n * sizeof(T)))) return st;
    if ((st = dev_alloc(h, &d.tau, n * sizeof(T)))) return st;
    if ((st = dev_alloc(h, &d.spec, n * sizeof(T)))) return st;   // n1/2 * n2 complex
    if ((st = dev_alloc(h, &d.spec2, n * sizeof(T)))) return st;
    const size_t nk = (size_t)(p.n1 / 2 + 1) * (p.n2 / 2 + 1);
    if ((st = dev_alloc(h, &d.Kh, nk * sizeof(T)))) return st;
    if ((st = dev_alloc(h, &d.tw1, (size_t)p.n1 * 2 * sizeof(T)))) return st;
    if ((st = dev_alloc(h, &d.tw2, (size_t)p.n2 * 2 * sizeof(T)))) return st;
    if ((st = dev_alloc(h, (void**)&d.row_partials, (size_t)d.geom.row_blocks * sizeof(double)))) return st;
    d.red_blocks = red_blocks_for(n);
    if ((st = dev_alloc(h, (void**)&d.red, (size_t)6 * d.red_blocks * sizeof(double)))) return st;
    if ((st = dev_alloc(h, (void**)&d.sc, sizeof(fdm_dev_scalars)))) return st;
    CK(cudaMemsetAsync(d.sc, 0, sizeof(fdm_dev_scalars), h->stream));
    if ((st = upload_twiddles<T>(h, d.tw1, p.n1))) return st;
    if ((st = upload_twiddles<T>(h, d.tw2, p.n2))) return st;
    // layer weights |chi-hat(k3)|^2, k3 in [0, nz/2] (Sec. 3.2.1 layer of nh voxels)
    std::vector<double> w3((size_t)p.nz / 2 + 1);
    for (int k3 = 0; k3 <= p.nz / 2; ++k3) {
        if (k3 == 0) { w3[k3] = (double)p.nh * p.nh; continue; }
        double sn = std::sin(kPi * (double)k3 * p.nh / p.nz), sd = std::sin(kPi * (double)k3 / p.nz);
        w3[k3] = (sn * sn) / (sd * sd);
    }
    void* dw3 = nullptr;
    void* dK64 = nullptr;
    if ((st = dev_alloc(h, &dw3, w3.size() * sizeof(double)))) return st;
    if ((st = dev_alloc(h, &dK64, nk * sizeof(double)))) return st;
    CK(cudaMemcpyAsync(dw3, w3.data(), w3.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    const double mu = p.E / (2.0 * (1.0 + p.nu));
    launch_kernel_table((double*)dK64, p.n1, p.n2, p.nz, p.nh, mu, p.nu, (const double*)dw3, h->stream);
    CK(cudaGetLastError());
    launch_convert<T>((const double*)dK64, (T*)d.Kh, nk, 0.0, h->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
    // release the create-time temporaries
    for (void* q : {dw3, dK64}) {
        cudaFree(q);
        for (size_t i = 0; i < h->owned.size(); ++i)
            if (h->owned[i] == q) { h->owned.erase(h->owned.begin() + i); break; }
    }
    return FDM_OK;
}

fdm_status reset_scalars(fdm_handle* h, double mean) {
    fdm_dev_scalars s;
    std::memset(&s, 0, sizeof(s));
    s.phi_ref = h->d.phi_ref_host;
    s.mean_up13 = mean;
    host_loading(h->d.p, 0, mean, &s.eps_bar13, &s.sigma_bar13);
    CK(cudaMemcpyAsync(h->d.sc, &s, sizeof(s), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->cur = 0;
    h->next_phase = 0;
    h->has_state = true;
    return FDM_OK;
}

// upload a host FP64 field into a device buffer of the handle's type (minus offset)
fdm_status upload_field(fdm_handle* h, void* dst, const double* src, double offset) {
    if (!h->mixed) {
        if (offset == 0.0) {
            CK(cudaMemcpyAsync(dst, src, h->n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            return FDM_OK;
        }
        std::vector<double> t(h->n);
        for (size_t i = 0; i < h->n; ++i) t[i] = src[i] - offset;
        CK(cudaMemcpyAsync(dst, t.data(), h->n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        return FDM_OK;
    }
    std::vector<float> t(h->n);
    for (size_t i = 0; i < h->n; ++i) t[i] = (float)(src[i] - offset);
    CK(cudaMemcpyAsync(dst, t.data(), h->n * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return FDM_OK;
}

fdm_status download_field(fdm_handle* h, double* dst, const void* src, double offset) {
    if (!h->mixed) {
        CK(cudaMemcpyAsync(dst, src, h->n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        if (offset != 0.0)
            for (size_t i = 0; i < h->n; ++i) dst[i] += offset;
        return FDM_OK;
    }
    std::vector<float> t(h->n);
    CK(cudaMemcpyAsync(t.data(), src, h->n * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (size_t i = 0; i < h->n; ++i) dst[i] = (double)t[i] + offset;
    return FDM_OK;
}

fdm_status read_scalars(fdm_handle* h, fdm_dev_scalars* s) {
    CK(cudaMemcpyAsync(s, h->d.sc, sizeof(*s), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return FDM_OK;
}

fdm_status fill_info(fdm_handle* h, fdm_step_info* info) {
    fdm_dev_scalars s;
    fdm_status st = read_scalars(h, &s);
    if (st) return st;
    Dev& d = h->d;
    const void* phi = d.phi[h->cur];
    if (h->mixed) launch_alpha_sums<float>(d, (const float*)phi, d.red, d.red_blocks, h->stream);
    else launch_alpha_sums<double>(d, (const double*)phi, d.red, d.red_blocks, h->stream);
    CK(cudaGetLastError());
    std::vector<double> part((size_t)6 * d.red_blocks);
    CK(cudaMemcpyAsync(part.data(), d.red, part.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    double sums[6];
    std::vector<double> col(d.red_blocks);
    for (int q = 0; q < 6; ++q) {
        for (int b = 0; b < d.red_blocks; ++b) col[b] = part[6 * b + q];
        sums[q] = ksum(col.data(), col.size());
    }
    std::memset(info, 0, sizeof(*info));
    info->step = s.step;
    info->t = s.t;
    info->dt = s.dt;
    info->max_abs_v0 = s.max_abs_v0;
    info->mean_up13 = s.phi_ref + sums[5] / (double)h->n;
    host_loading(d.p, s.step, info->mean_up13, &info->eps_bar13, &info->sigma_bar13);
    info->sum_a12_pos = sums[0];
    info->sum_a12_neg = sums[1];
    info->sum_a11_pos = sums[2];
    info->sum_a11_neg = sums[3];
    info->sum_abs_alpha = sums[4];
    info->status = s.status;
    return FDM_OK;
}

template <typename T>
fdm_status ensure_readout(fdm_handle* h) {
    for (int i = 0; i < 4; ++i)
        if (!h->rd[i]) {
            fdm_status st = dev_alloc(h, &h->rd[i], h->n * sizeof(T));
            if (st) return st;
        }
    return FDM_OK;
}

template <typename T>
fdm_status read_fields_impl(fdm_handle* h, uint32_t mask, double* up13, double* a11, double* a12, double* tau,
                            double* v1, double* v2) {
    Dev& d = h->d;
    const T* phi = (const T*)d.phi[h->cur];
    fdm_status st;
    if (mask & FDM_FIELD_UP13)
        if ((st = download_field(h, up13, phi, d.phi_ref_host))) return st;
    if (mask & FDM_FIELD_TAU13)
        if ((st = download_field(h, tau, d.tau, 0.0))) return st;
    if (mask & (FDM_FIELD_ALPHA11 | FDM_FIELD_ALPHA12 | FDM_FIELD_V1 | FDM_FIELD_V2)) {
        if ((st = ensure_readout<T>(h))) return st;
        launch_alpha<T>(d, phi, (T*)h->rd[0], (T*)h->rd[1], h->stream);
        CK(cudaGetLastError());
        if (mask & FDM_FIELD_ALPHA11)
            if ((st = download_field(h, a11, h->rd[0], 0.0))) return st;
        if (mask & FDM_FIELD_ALPHA12)
            if ((st = download_field(h, a12, h->rd[1], 0.0))) return st;
        if (mask & (FDM_FIELD_V1 | FDM_FIELD_V2)) {
            launch_velocity<T>(d, (const T*)h->rd[0], (const T*)h->rd[1], (const T*)d.tau, phi, (T*)h->rd[2],
                               (T*)h->rd[3], h->stream);
            CK(cudaGetLastError());
            if (mask & FDM_FIELD_V1)
                if ((st = download_field(h, v1, h->rd[2], 0.0))) return st;
            if (mask & FDM_FIELD_V2)
                if ((st = download_field(h, v2, h->rd[3], 0.0))) return st;
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
    p->theta = 1.0;
    p->cfl = 0.5;
    p->dt_max = 0.0;
    p->loading_mode = FDM_LOAD_STRESS;
    p->time_level = FDM_T_MIDPOINT;
    p->precision = FDM_FP64;
}

size_t fdm_device_bytes(const fdm_params* p) {
    if (!valid(p)) return 0;
    size_t n = (size_t)p->n1 * p->n2, e = elt(p);
    size_t nk = (size_t)(p->n1 / 2 + 1) * (p->n2 / 2 + 1);
    return 5 * n * e + nk * e + (size_t)(p->n1 + p->n2) * 2 * e + 64 * 1024;
}

fdm_status fdm_create(const fdm_params* p, void* stream, fdm_handle** out) {
    if (!out) return FDM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!valid(p)) return FDM_ERR_INVALID_ARG;
    fdm_handle* h = new (std::nothrow) fdm_handle();
    if (!h) return FDM_ERR_OOM;
    h->d.p = *p;
    if (h->d.p.nz == 0) h->d.p.nz = p->n1;
    h->stream = (cudaStream_t)stream;
    h->cur = 0;
    h->has_state = false;
    h->mixed = p->precision == FDM_MIXED;
    h->n = (size_t)p->n1 * p->n2;
    h->d.phi_ref_host = 0.0;
    fdm_status st = h->mixed ? create_impl<float>(h) : create_impl<double>(h);
    if (st != FDM_OK) {
        fdm_destroy(h);
        return st;
    }
    *out = h;
    return FDM_OK;
}

fdm_status fdm_set_plastic_distortion(fdm_handle* h, const double* up13) {
    if (!h || !up13) return FDM_ERR_INVALID_ARG;
    double mean = ksum(up13, h->n) / (double)h->n;
    if (!std::isfinite(mean)) return FDM_ERR_INVALID_ARG;
    h->d.phi_ref_host = h->mixed ? mean : 0.0;
    fdm_status st = upload_field(h, h->d.phi[0], up13, h->d.phi_ref_host);
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
    Dev& d = h->d;
    fdm_status st;
    // stage alpha in the two state buffers (the old state is being replaced)
    if ((st = upload_field(h, d.phi[0], a11, 0.0))) return st;
    if ((st = upload_field(h, d.phi[1], a12, 0.0))) return st;
    double phi_ref = h->mixed ? mean_up13 : 0.0;
    const int nblk = d.red_blocks;
    if (h->mixed)
        launch_curl_inverse<float>(d, (const float*)d.phi[0], (const float*)d.phi[1], (float*)d.phi[0], mean_up13,
                                   phi_ref, d.red, nblk, h->stream);
    else
        launch_curl_inverse<double>(d, (const double*)d.phi[0], (const double*)d.phi[1], (double*)d.phi[0],
                                    mean_up13, phi_ref, d.red, nblk, h->stream);
    CK(cudaGetLastError());
    std::vector<double> part((size_t)2 * nblk);
    CK(cudaMemcpyAsync(part.data(), d.red, part.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    double num = 0.0, den = 0.0;
    for (int b = 0; b < nblk; ++b) { num += part[2 * b]; den += part[2 * b + 1]; }
    double res = den > 0.0 ? std::sqrt(num / den) : 0.0;
    if (div_residual) *div_residual = res;
    d.phi_ref_host = phi_ref;
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
    CK(cudaMemcpyAsync(h->d.sc, &s, sizeof(s), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return FDM_OK;
}

fdm_status fdm_static_solve(fdm_handle* h) {
    if (!h) return FDM_ERR_INVALID_ARG;
    if (!h->has_state || h->next_phase != 0) return FDM_ERR_STATE;
    Dev& d = h->d;
    if (h->mixed) launch_static<float>(d, (const float*)d.phi[h->cur], h->stream);
    else launch_static<double>(d, (const double*)d.phi[h->cur], h->stream);
    CK(cudaGetLastError());
    // the stencil kernel normally clears the running max; no step follows here
    CK(cudaMemsetAsync(&d.sc->vmax_bits, 0, sizeof(unsigned long long), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return FDM_OK;
}

fdm_status fdm_enqueue_steps(fdm_handle* h, int32_t nsteps) {
    if (!h || nsteps < 0) return FDM_ERR_INVALID_ARG;
    if (!h->has_state || h->next_phase != 0) return FDM_ERR_STATE;
    Dev& d = h->d;
    for (int32_t i = 0; i < nsteps; ++i) {
        int nx = h->cur ^ 1;
        if (h->mixed) launch_step<float>(d, (const float*)d.phi[h->cur], (float*)d.phi[nx], h->stream);
        else launch_step<double>(d, (const double*)d.phi[h->cur], (double*)d.phi[nx], h->stream);
        h->cur = nx;
    }
    CK(cudaGetLastError());
    return FDM_OK;
}

fdm_status fdm_enqueue_phase(fdm_handle* h, int32_t phase) {
    if (!h || phase < 0 || phase >= kKernelsPerStep) return FDM_ERR_INVALID_ARG;
    if (!h->has_state || phase != h->next_phase) return FDM_ERR_STATE;
    Dev& d = h->d;
    int nx = h->cur ^ 1;
    if (h->mixed) launch_phase<float>(d, phase, (const float*)d.phi[h->cur], (float*)d.phi[nx], h->stream);
    else launch_phase<double>(d, phase, (const double*)d.phi[h->cur], (double*)d.phi[nx], h->stream);
    CK(cudaGetLastError());
    h->next_phase = phase + 1;
    if (h->next_phase == kKernelsPerStep) {
        h->next_phase = 0;
        h->cur = nx;
    }
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
        if ((st = fill_info(h, info))) return st;
        return info->status ? (fdm_status)info->status : FDM_OK;
    }
    fdm_dev_scalars s;
    if ((st = read_scalars(h, &s))) return st;
    return s.status ? (fdm_status)s.status : FDM_OK;
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
    return h->mixed ? read_fields_impl<float>(h, mask, up13, a11, a12, tau, v1, v2)
                    : read_fields_impl<double>(h, mask, up13, a11, a12, tau, v1, v2);
}

fdm_status fdm_get_info(fdm_handle* h, fdm_step_info* info) {
    if (!h || !info) return FDM_ERR_INVALID_ARG;
    if (!h->has_state) return FDM_ERR_STATE;
    return fill_info(h, info);
}

int32_t fdm_kernels_per_step(const fdm_handle* h) {
    (void)h;
    return kKernelsPerStep;
}

void fdm_destroy(fdm_handle* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    for (void* q : h->owned) cudaFree(q);
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
