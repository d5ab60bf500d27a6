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

// The scratch: 692,992 bytes.  In host code this name is only a stand-in for the device
// symbol; kernels get its device address from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];
static_assert(kScratchDoubles * sizeof(double) == 692992, "the size stated in include/fdm.h");

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};
bool g_ready[kMaxDevices] = {};

bool pow2_between(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

// Once per device, with that device current: resolve the scratch address and set the
// kernels' shared-memory limits.
fdm_status setup_device(int dev, double** out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_ready[dev]) {
        // resolving the symbol loads the library's device code onto this device if it is not
        // there yet (CUDA loads modules lazily by default): that allocation by the driver is
        // why the first call should come before the caller commits its memory
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e == cudaSuccess && ptr == nullptr) e = cudaErrorInvalidSymbol;
        if (e == cudaSuccess) e = configure_kernels<double>();
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? FDM_ERR_OOM : FDM_ERR_DEVICE;
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
    if (!p || !d_up13 || !d_tau13) return FDM_ERR_INVALID_ARG;
    if (((uintptr_t)d_up13 | (uintptr_t)d_tau13) & 15u) return FDM_ERR_INVALID_ARG;   // 16-byte aligned
    if (p->precision != FDM_FP64 || !std::isfinite(sigma_bar13)) return FDM_ERR_INVALID_ARG;
    const int nz = p->nz == 0 ? p->n1 : p->nz;
    if (!pow2_between(p->n1, 16, 1 << 30) || !pow2_between(p->n2, 16, 1 << 30)) return FDM_ERR_INVALID_ARG;
    if (p->n1 > kMaxSide || p->n2 > kMaxSide || nz > kMaxNz) return FDM_ERR_TOO_LARGE;
    if (nz < 1 || p->nh < 1 || p->nh > nz) return FDM_ERR_INVALID_ARG;
    if (!(p->E > 0.0) || !(p->nu > -1.0 && p->nu < 0.5) || !(p->dx > 0.0) || !std::isfinite(p->dx) ||
        !std::isfinite(p->E))
        return FDM_ERR_INVALID_ARG;
    {   // the output is written while the input is still being read: the arrays may not overlap
        const size_t n = (size_t)p->n1 * p->n2;
        const uintptr_t a = (uintptr_t)d_up13, b = (uintptr_t)d_tau13;
        if (a < b + n * sizeof(double) && b < a + n * sizeof(double)) return FDM_ERR_INVALID_ARG;
    }

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
    // the same table routines as the handle path (fdm_create)
    launch_twiddle_tables<double>(base + kOffTw1, p->n1, base + kOffPt1, p->n1 / 2, s);
    launch_twiddle_tables<double>(base + kOffTw2, p->n2, base + kOffPt2, p->n2, s);
    launch_layer_weights(base + kOffW3, nz, p->nh, s);
    const double mu = p->E / (2.0 * (1.0 + p->nu));
    launch_kernel_table(base + kOffK, p->n1, p->n2, nz, p->nh, mu, p->nu, base + kOffW3, s);
    launch_static<double>(d, s);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? FDM_ERR_OOM : FDM_ERR_DEVICE;
    return FDM_OK;
}
