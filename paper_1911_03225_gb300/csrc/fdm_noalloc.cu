// fdm_noalloc.cu -- static solve that allocates no device memory.
//
// Some callers cannot let a library allocate: a serving process that has already handed
// its whole HBM budget to request slots, or an embedding that only permits allocations
// through its own pool.  fdm_static_solve_noalloc serves them: the caller passes its own
// device input and output, and every intermediate (half spectrum, layer kernel table,
// twiddles, partial sums, scalars) lives in one file-scope device array of fixed size.
// The array exists on every GPU that loads this library and stays there until exit.
#include <cmath>
#include <mutex>

#include "fdm_device.cuh"
#include "fdm_internal.h"

namespace fdm {
namespace {

// Largest grid accepted: n1, n2 <= 256 (65536 cells), cell depth nz <= 4096.
constexpr int kMaxSide = 256;
constexpr int kMaxNz = 4096;
constexpr size_t kAlignD = 32;  // 256 bytes in doubles
constexpr size_t round_up(size_t v) { return (v + kAlignD - 1) / kAlignD * kAlignD; }
constexpr size_t kOffSpec = 0;                                              // n1*n2 doubles
constexpr size_t kOffK = kOffSpec + round_up((size_t)kMaxSide * kMaxSide);  // (n1/2+1)(n2/2+1)
constexpr size_t kOffTw1 = kOffK + round_up((size_t)(kMaxSide / 2 + 1) * (kMaxSide / 2 + 1));
constexpr size_t kOffTw2 = kOffTw1 + round_up((size_t)2 * kMaxSide);
constexpr size_t kOffPt1 = kOffTw2 + round_up((size_t)2 * kMaxSide);  // pass tables (< side entries)
constexpr size_t kOffPt2 = kOffPt1 + round_up((size_t)2 * kMaxSide);
constexpr size_t kOffW3 = kOffPt2 + round_up((size_t)2 * kMaxSide);
constexpr size_t kOffPart = kOffW3 + round_up((size_t)kMaxNz / 2 + 1);
constexpr size_t kOffSc = kOffPart + round_up((size_t)kMaxSide);
constexpr size_t kScratchDoubles = kOffSc + round_up(sizeof(fdm_dev_scalars) / sizeof(double) + 1);

// The scratch (about 710 KB).  In host code this name is only a stand-in for the device
// symbol; kernels get its device address from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};
bool g_ready[kMaxDevices] = {};

// twiddles exp(-2 pi i m / n) and the layer weights |chi-hat(k3)|^2 (Sec. 3.2.1)
__global__ void noalloc_tables_kernel(double* tw1, int n1, double* tw2, int n2, double* w3, int nz, int nh) {
    const int top = max(max(n1, n2), nz / 2 + 1);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < top; i += gridDim.x * blockDim.x) {
        double s, c;
        if (i < n1) { sincospi(2.0 * (double)i / (double)n1, &s, &c); tw1[2 * i] = c; tw1[2 * i + 1] = -s; }
        if (i < n2) { sincospi(2.0 * (double)i / (double)n2, &s, &c); tw2[2 * i] = c; tw2[2 * i + 1] = -s; }
        if (i <= nz / 2) {
            if (i == 0) {
                w3[0] = (double)nh * (double)nh;
            } else {
                double sn = sinpi((double)i * (double)nh / (double)nz), sd = sinpi((double)i / (double)nz);
                w3[i] = (sn * sn) / (sd * sd);
            }
        }
    }
}

// per-pass twiddle tables of an L-point transform (entry layout as in pass_table_len)
__global__ void noalloc_pass_table_kernel(double* pt, int L) {
    const int len = pass_table_len(L);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) {
        int off = 0, Ns = 1, R = 8;
        while (true) {
            R = (Ns * 8 <= L) ? 8 : (Ns * 4 == L ? 4 : 2);
            if (i < off + (R - 1) * Ns) break;
            off += (R - 1) * Ns;
            Ns *= R;
        }
        const int r = (i - off) / Ns + 1, k = (i - off) % Ns;
        double sn, cs;
        sincospi(2.0 * (double)r * (double)k / ((double)Ns * R), &sn, &cs);
        pt[2 * i] = cs;
        pt[2 * i + 1] = -sn;
    }
}

bool pow2_between(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

// Once per device, with that device current: resolve the scratch address and set the
// kernels' shared-memory limits.
fdm_status setup_device(int dev, double** out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_ready[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            return FDM_ERR_DEVICE;
        }
        if (configure_kernels<double>() != cudaSuccess) {
            cudaGetLastError();
            return FDM_ERR_DEVICE;
        }
        g_scratch_ptr[dev] = static_cast<double*>(ptr);
        g_ready[dev] = true;
    }
    *out = g_scratch_ptr[dev];
    return FDM_OK;
}

}  // namespace
}  // namespace fdm

using namespace fdm;

extern "C" fdm_status fdm_static_solve_noalloc(const fdm_params* p, double sigma_bar13, const double* d_up13,
                                               double* d_tau13, void* stream) {
    if (!p || !d_up13 || !d_tau13 || d_up13 == d_tau13) return FDM_ERR_INVALID_ARG;
    if (p->precision != FDM_FP64 || !std::isfinite(sigma_bar13)) return FDM_ERR_INVALID_ARG;
    const int nz = p->nz == 0 ? p->n1 : p->nz;
    if (!pow2_between(p->n1, 16, 1 << 30) || !pow2_between(p->n2, 16, 1 << 30)) return FDM_ERR_INVALID_ARG;
    if (p->n1 > kMaxSide || p->n2 > kMaxSide || nz > kMaxNz) return FDM_ERR_TOO_LARGE;
    if (nz < 1 || p->nh < 1 || p->nh > nz) return FDM_ERR_INVALID_ARG;
    if (!(p->E > 0.0) || !(p->nu > -1.0 && p->nu < 0.5) || !(p->dx > 0.0)) return FDM_ERR_INVALID_ARG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return FDM_ERR_DEVICE;
    }
    double* base = nullptr;
    fdm_status st = setup_device(dev, &base);
    if (st != FDM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;

    Dev d{};
    d.count = 1;
    d.gated = 0;
    d.p = *p;
    d.p.nz = nz;
    d.p.velocity_mode = FDM_V_PRESCRIBED;   // tau13 only: no celerity law needed
    d.p.loading_mode = FDM_LOAD_STRESS;     // mean of tau13 = the given macroscopic stress
    d.p.sigma_bar13 = sigma_bar13;
    d.geom = geometry<double>(p->n1, p->n2);
    d.phi[0] = const_cast<double*>(d_up13);   // buffer 0 is current (scalars start at zero)
    d.phi[1] = nullptr;
    d.tau = d_tau13;
    d.spec = base + kOffSpec;
    d.spec2 = nullptr;
    d.Kh = base + kOffK;
    d.tw1 = base + kOffTw1;
    d.tw2 = base + kOffTw2;
    d.pt1 = base + kOffPt1;
    d.pt2 = base + kOffPt2;
    d.row_partials = base + kOffPart;
    d.red = nullptr;
    d.red_blocks = 0;
    d.sc = reinterpret_cast<fdm_dev_scalars*>(base + kOffSc);
    d.phi_ref_host = 0.0;

    // The scratch keeps the previous call's contents: the scalars must start at zero.
    if (cudaMemsetAsync(d.sc, 0, sizeof(fdm_dev_scalars), s) != cudaSuccess) {
        cudaGetLastError();
        return FDM_ERR_DEVICE;
    }
    noalloc_tables_kernel<<<8, 256, 0, s>>>(base + kOffTw1, p->n1, base + kOffTw2, p->n2, base + kOffW3, nz, p->nh);
    noalloc_pass_table_kernel<<<1, 256, 0, s>>>(base + kOffPt1, p->n1 / 2);
    noalloc_pass_table_kernel<<<1, 256, 0, s>>>(base + kOffPt2, p->n2);
    const double mu = p->E / (2.0 * (1.0 + p->nu));
    launch_kernel_table(base + kOffK, p->n1, p->n2, nz, p->nh, mu, p->nu, base + kOffW3, s);
    launch_static<double>(d, s);
    if (cudaGetLastError() != cudaSuccess) return FDM_ERR_DEVICE;
    return FDM_OK;
}
