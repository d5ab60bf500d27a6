// fdm_kernels.cu -- CUDA kernels (sm_103a) of the FDM layer-case time step
// (arXiv 1911.03225, Sec. 3.1.1 splitting; Sec. 3.1.2 static problem by FFT;
// Sec. 3.2.2-3.2.3 Kurganov-Noelle-Petrova transport).
//
// Data layout in HBM (x1 fastest):
//   phi   [n2][n1]            U13 (FP64, or FP32 minus an FP64 reference in mixed mode)
//   tau   [n2][n1]            layer-averaged shear stress of the last static solve
//   spec  [n1/2][n2] complex  packed half spectrum, TRANSPOSED: column kx holds, for all
//                             x2, the row transform's coefficient kx; kx = 0 packs
//                             X(0) + i X(n1/2) (both real for a real row)
//   Kh    [n1/2+1][n2/2+1]    layer Green kernel K(kx, |ky|) (even in both indices)
//
// One step = row_forward (R2C of every row, transposed store) -> col_pass (FFT along x2,
// multiply by K, inverse FFT along x2) -> row_inverse (C2R, tau and max|v0|) -> knp_step.
#include <type_traits>

#include "fdm_device.cuh"
#include "fdm_internal.h"

namespace fdm {

// ------------------------------------------------------------------ small helpers
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// block-wide sum, fixed order (deterministic); result valid in thread 0
__device__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) for (int i = 0; i < nw; ++i) r += red[i];
    __syncthreads();
    return r;
}
// max of non-negative values, NaN-propagating through the bit order (NaN > +inf)
__device__ __forceinline__ unsigned long long abs_bits(double v) {
    return (unsigned long long)__double_as_longlong(fabs(v));
}

__device__ __forceinline__ void loading_state(const fdm_params& p, long long step, double t, double mean,
                                              double* eps, double* sig) {
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


// Instance addressing of the step kernels: a launch covers `count` instances (grid y, or z
// for the stencil).  sc == nullptr marks a set-up launch (one instance, buffer 0, always
// runs).  Otherwise instance i reads U13 from buffer sc[i].cur, and with gating on it runs
// only while its step budget sc[i].steps_left is non-zero.  Read by thread 0 only and
// broadcast, so that every thread of a block sees the same values.
struct InstCtl {
    fdm_dev_scalars* sc;
    int gated;
};

__device__ __forceinline__ void inst_state(const InstCtl& c, int inst, int* run, int* cur) {
    int r = 1, k = 0;
    if (c.sc) {
        const fdm_dev_scalars* si = c.sc + inst;
        k = si->cur;
        if (c.gated && si->steps_left == 0) r = 0;
    }
    *run = r;
    *cur = k;
}

// Neumaier step s + x with compensation c (FP64; the magnitude test on bit patterns)
__device__ __forceinline__ void neumaier_add(double& s, double& c, double x) {
    const double t = s + x;
    c += ((ubits(s) & kMagBits) >= (ubits(x) & kMagBits)) ? (s - t) + x : (x - t) + s;
    s = t;
}

// one element global -> shared without passing through registers (4, 8 or 16 bytes)
template <typename T> __device__ __forceinline__ void copy_async(T* smem_dst, const T* gmem_src) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8 || sizeof(T) == 16, "4-, 8- or 16-byte elements");
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(gmem_src), "n"(sizeof(T)) : "memory");
}
// waits for all of this thread's asynchronous copies (the block barrier that follows makes
// every thread's copies visible to all)
__device__ __forceinline__ void copy_async_wait_all() {
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Thread and residency bounds of the FFT kernels.  The FP32 kernels are latency bound: a
// block of at most 512 threads with three resident per SM caps them at 40 registers, which
// keeps 48 warps per SM instead of 32 (no spills).
template <typename T> struct FftBounds { static constexpr int threads = 1024, minb = 1; };
template <> struct FftBounds<float> { static constexpr int threads = 512, minb = 3; };

// The FP32 transforms read their pass twiddles from shared memory, staged once per block
// behind the data (visible after the block's next barrier): those kernels are latency bound,
// and a shared load waits less than a global one.  Other types keep the global tables.
template <typename T> __host__ __device__ __forceinline__ size_t staged_twiddle_bytes(int L) {
    return std::is_same<T, float>::value ? (size_t)pass_table_len(L) * sizeof(cpx<T>) : 0;
}
// The FP32 transforms pass between two shared buffers (one barrier per pass); the others
// transform in place in one.  Buffers of the block's sequences: fft_buffers<T>() x nseq x ld.
template <typename T> __host__ __device__ constexpr int fft_buffers() { return std::is_same<T, float>::value ? 2 : 1; }
// the transform of the block's sequences in A (and the second buffer B for FP32); returns the
// buffer holding the result
template <int S, typename T>
__device__ __forceinline__ cpx<T>* block_fft(cpx<T>* A, cpx<T>* B, int L, int nseq, int ld, const cpx<T>* ptw) {
    if constexpr (fft_buffers<T>() == 2) {
        return smem_fft_pp<S>(A, B, L, nseq, ld, ptw);
    } else {
        smem_fft_ip<S>(A, L, nseq, ld, ptw);
        return A;
    }
}
template <typename T>
__device__ __forceinline__ const cpx<T>* stage_twiddles(const cpx<T>* pt, cpx<T>* slot, int L) {
    if constexpr (std::is_same<T, float>::value) {
        const int len = pass_table_len(L);
        for (int i = threadIdx.x; i < len; i += blockDim.x) copy_async(slot + i, pt + i);
        return slot;
    } else {
        return pt;
    }
}

// ------------------------------------------------------------------ row forward (R2C)
// grid: n2 / R blocks; block b handles rows [b R, b R + R).  Optional FP64 sum of each row
// (for <U13>), in an order fixed by the row alone, so that results do not depend on R.
// body of one block: rows [tile R, tile R + R) of instance inst (also run as a task of the
// persistent batched step)
template <typename T>
__device__ __forceinline__ void row_forward_body(const T* src0, const T* src1, cpx<T>* spec, int n1, int n2, int R,
                                                 const cpx<T>* __restrict__ tw1, const cpx<T>* __restrict__ pt1,
                                                 double* row_partials, InstCtl ctl, int tile, int inst) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_run, s_cur;
    
    if (threadIdx.x == 0) inst_state(ctl, inst, &s_run, &s_cur);
    __syncthreads();
    if (!s_run) return;
    const size_t nn = (size_t)n1 * n2;
    const T* src = (s_cur ? src1 : src0) + inst * nn;
    spec += inst * (nn / 2);
    if (row_partials) row_partials += (size_t)inst * n2;
    const int L = n1 >> 1;
    const int ld = padded_len(L);  // padded sequence stride (bank spread for the transposed store)
    cpx<T>* A = reinterpret_cast<cpx<T>*>(smem_raw);  // R * ld elements
    cpx<T>* B = A + R * ld;   // second buffer (FP32)
    const cpx<T>* ptw = stage_twiddles<T>(pt1, A + fft_buffers<T>() * R * ld, L);
    const int y0 = tile * R;
    const int lL = 31 - __clz(L), lR = 31 - __clz(R);  // powers of two
    const cpx<T>* src2 = reinterpret_cast<const cpx<T>*>(src) + (size_t)y0 * L;  // rows are contiguous
    const int total = R * L, step = blockDim.x;
    // every element (and the staged twiddles) by asynchronous copies, all in flight at once
    for (int e = threadIdx.x; e < total; e += step) copy_async(A + (e >> lL) * ld + swz(e & (L - 1)), src2 + e);
    copy_async_wait_all();
    __syncthreads();
    if (row_partials) {
        // one warp per row: lane l sums the pairs l, l + 32, ... (compensated, in the field's
        // type), then a fixed FP64 butterfly over the lanes
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int r = threadIdx.x >> 5; r < R; r += nw) {
            T acc = T(0), comp = T(0);
            for (int m = lane; m < L; m += 32) {
                const cpx<T> v = A[r * ld + swz(m)];
                T y = (v.x + v.y) - comp;
                T t = acc + y;
                comp = (t - acc) - y;
                acc = t;
            }
            const double rs = warp_sum((double)acc - (double)comp);
            if (lane == 0) row_partials[y0 + r] = rs;
        }
    }
    cpx<T>* F = block_fft<-1>(A, B, L, R, ld, ptw);
    // in place: a thread owns the pair (k, L - k), k < L/2, of one row; the cheap k = 0 item
    // also takes the middle k = L/2 (L >= 8)
    const int hq = L >> 1;
    for (int e = threadIdx.x; e < R * hq; e += blockDim.x) {
        const int r = e >> (lL - 1), k = e & (hq - 1);
        r2c_twist_pair(F + r * ld, F + r * ld, L, k, tw1);
        if (k == 0) r2c_twist_pair(F + r * ld, F + r * ld, L, hq, tw1);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < R * L; e += blockDim.x) {
        int kx = e >> lR, r = e & (R - 1);
        spec[(size_t)kx * n2 + y0 + r] = F[r * ld + swz(kx)];
    }
}

template <typename T>
__global__ void __launch_bounds__(FftBounds<T>::threads, FftBounds<T>::minb) row_forward_kernel(const T* src0, const T* src1, cpx<T>* spec,
                                                          int n1, int n2, int R,
                                                          const cpx<T>* __restrict__ tw1,
                                                          const cpx<T>* __restrict__ pt1,
                                                          double* row_partials, InstCtl ctl) {
    row_forward_body<T>(src0, src1, spec, n1, n2, R, tw1, pt1, row_partials, ctl, blockIdx.x, blockIdx.y);
}

// ------------------------------------------------------------------ column pass
// grid: (n1/2) / C blocks; block handles columns [b C, b C + C) of the transposed spectrum.
// Multiplier modes (all include the 1/(n1 n2) normalisation):
//   COL_K         tau-hat = K U-hat, DC = sigma_bar13 (block 0 computes <U13> and loading)
//   COL_DERIV1    alpha12-hat = i xi1 U-hat  (odd symbol, 0 at the x1 Nyquist index)
//   COL_DERIV2N   alpha11-hat = -i xi2 U-hat (odd symbol, 0 at the x2 Nyquist index)
//   COL_FWD       forward transform only (no normalisation)
//   COL_INV       inverse transform only
//   COL_SYM       stress component on a plane of the 3-D cell: the quarter table Kh holds
//                 |symbol| for kx, ky >= 0 (normalisation folded in); the symbol is i times
//                 it when sym_imag, and changes sign with ky when sym_odd2 (the sign in kx
//                 never enters: kx >= 0 in the half spectrum); DC is zero
constexpr int kRedLanes = 256;  // lanes of the <U13> reduction in the column kernel
enum ColMode { COL_K = 0, COL_DERIV1 = 1, COL_DERIV2N = 2, COL_FWD = 3, COL_INV = 4, COL_SYM = 5 };

template <typename T>
struct ColArgs {
    fdm_params p;
    int mode;
    const double* row_partials;  // COL_K: per-row sums of U13 (nparts = n2 entries)
    int nparts;
    fdm_dev_scalars* sc;         // COL_K: scalars of instance 0 (block 0 writes mean/eps/sigma)
    int gated;                   // COL_K: honour the instances' step budgets
    T scl;                       // 1 / (n1 n2)
    T xi1_unit, xi2_unit;        // 2 pi / (n dx): xi = k~ * unit
    int sym_odd2, sym_imag;      // COL_SYM: symbol odd in xi2; symbol imaginary
};

template <typename T>
__device__ __forceinline__ cpx<T> col_multiplier(const ColArgs<T>& a, const T* __restrict__ Kh, int kxi,
                                                 int ky, int n1, int n2) {
    // kxi in [0, n1/2]; ky in [0, n2)
    if (a.mode == COL_K) {   // the table carries the 1/(n1 n2) normalisation
        int kyf = ky <= n2 / 2 ? ky : n2 - ky;
        return mk(Kh[(size_t)kxi * (n2 / 2 + 1) + kyf], T(0));
    }
    if (a.mode == COL_SYM) {
        int kyf = ky <= n2 / 2 ? ky : n2 - ky;
        T v = Kh[(size_t)kxi * (n2 / 2 + 1) + kyf];
        if (a.sym_odd2 && ky > n2 / 2) v = -v;
        return a.sym_imag ? mk(T(0), v) : mk(v, T(0));
    }
    if (a.mode == COL_DERIV1) {
        if (2 * kxi == n1) return mk(T(0), T(0));
        return mk(T(0), T(kxi) * a.xi1_unit * a.scl);
    }
    // COL_DERIV2N
    if (2 * ky == n2) return mk(T(0), T(0));
    int kys = ky <= n2 / 2 ? ky : ky - n2;
    return mk(T(0), -(T(kys) * a.xi2_unit) * a.scl);
}

// the symbol applied to one coefficient: real (K) or imaginary (derivatives), so two
// multiplications rather than a general complex product
template <typename T>
__device__ __forceinline__ cpx<T> col_apply(const ColArgs<T>& a, const T* __restrict__ Kh, int kxi, int ky,
                                            int n1, int n2, cpx<T> z) {
    const cpx<T> m = col_multiplier<T>(a, Kh, kxi, ky, n1, n2);
    if (a.mode == COL_K || (a.mode == COL_SYM && !a.sym_imag)) return mk(m.x * z.x, m.x * z.y);
    return mk(-(m.y * z.y), m.y * z.x);
}

// body of one block: columns [tile C, tile C + C) of instance inst
template <typename T>
__device__ __forceinline__ void col_pass_body(const cpx<T>* in, cpx<T>* out, int n1, int n2, int C,
                                              const cpx<T>* __restrict__ pt2, const T* __restrict__ Kh,
                                              ColArgs<T> a, int tile, int inst) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ld = padded_len(n2);
    const int ln2 = 31 - __clz(n2);
    cpx<T>* A = reinterpret_cast<cpx<T>*>(smem_raw);
    __shared__ double s_sigma;
    __shared__ double s_red[kRedLanes];
    __shared__ int s_run, s_cur;
    
    if (threadIdx.x == 0) {
        InstCtl ctl{a.mode == COL_K ? a.sc : nullptr, a.gated};
        inst_state(ctl, inst, &s_run, &s_cur);
    }
    __syncthreads();
    if (!s_run) return;
    cpx<T>* B = A + C * ld;   // second buffer (FP32)
    const cpx<T>* ptw = stage_twiddles<T>(pt2, A + fft_buffers<T>() * C * ld, n2);
    const size_t half_n = (size_t)n1 * n2 / 2;
    in += inst * half_n;
    out += inst * half_n;
    fdm_dev_scalars* sci = a.sc ? a.sc + inst : nullptr;
    const double* parts = a.row_partials ? a.row_partials + (size_t)inst * a.nparts : nullptr;
    const int kx0 = tile * C;
    const cpx<T>* src = in + (size_t)kx0 * n2;
    {
        const int total = C * n2, step = blockDim.x;
        for (int e = threadIdx.x; e < total; e += step) copy_async(A + (e >> ln2) * ld + swz(e & (n2 - 1)), src + e);
        copy_async_wait_all();
    }
    if (a.mode == COL_K && kx0 == 0) {
        // <U13> from the row sums, then the loading state of this step (Sec. 5.1).  The
        // order is fixed by n2 alone: kRedLanes compensated lane sums over a stride, then a
        // fixed tree (results do not depend on the launch shape)
        for (int v = threadIdx.x; v < kRedLanes; v += blockDim.x) {
            double s = 0.0, c = 0.0;
            for (int i = v; parts && i < a.nparts; i += kRedLanes) neumaier_add(s, c, parts[i]);
            s_red[v] = s + c;
        }
        __syncthreads();
        double tot = 0.0;
        if (threadIdx.x < 32) {
            double s = 0.0, c = 0.0;
            for (int v = threadIdx.x; v < kRedLanes; v += 32) neumaier_add(s, c, s_red[v]);
            tot = warp_sum(s + c);
        }
        if (threadIdx.x == 0) {
            double mean = parts ? sci->phi_ref + tot / ((double)n1 * (double)n2) : sci->mean_up13;
            double eps, sig;
            loading_state(a.p, sci->step, sci->t, mean, &eps, &sig);
            sci->mean_up13 = mean;
            sci->eps_bar13 = eps;
            sci->sigma_bar13 = sig;
            s_sigma = sig;
        }
    }
    __syncthreads();
    cpx<T>* F = A;
    if (a.mode != COL_INV) F = block_fft<-1>(A, B, n2, C, ld, ptw);
    cpx<T>* G = (F == A) ? B : A;   // the other buffer
    if (a.mode == COL_K || a.mode == COL_DERIV1 || a.mode == COL_DERIV2N || a.mode == COL_SYM) {
        // in place: a thread owns the pair (ky, n2 - ky), ky < n2/2, of one column, and the
        // ky = 0 item also the middle ky = n2/2
        const int hq = n2 >> 1;
        auto item = [&](int c, int ky) {
            const int kyr = (n2 - ky) & (n2 - 1);
            const int kx = kx0 + c;
            cpx<T>* col = F + c * ld;
            const cpx<T> z = col[swz(ky)], zr = col[swz(kyr)];
            cpx<T> o, orr;
            if (kx > 0) {
                o = col_apply<T>(a, Kh, kx, ky, n1, n2, z);
                orr = col_apply<T>(a, Kh, kx, kyr, n1, n2, zr);
            } else {
                // packed column: z = C0 + i CN (C0, CN transforms of the real columns kx = 0
                // and kx = n1/2); multiply each by its own symbol and repack:
                // out(ky) = (m0 + mN)/2 z(ky) + (m0 - mN)/2 conj(z(-ky))
                cpx<T> m0 = col_multiplier<T>(a, Kh, 0, ky, n1, n2);
                cpx<T> mN = col_multiplier<T>(a, Kh, n1 / 2, ky, n1, n2);
                o = cmul(scale(m0 + mN, T(0.5)), z) + cmul(scale(m0 - mN, T(0.5)), conj(zr));
                cpx<T> m0r = col_multiplier<T>(a, Kh, 0, kyr, n1, n2);
                cpx<T> mNr = col_multiplier<T>(a, Kh, n1 / 2, kyr, n1, n2);
                orr = cmul(scale(m0r + mNr, T(0.5)), zr) + cmul(scale(m0r - mNr, T(0.5)), conj(z));
                if (ky == 0 && a.mode == COL_K) o.x = T(s_sigma);  // macroscopic stress
            }
            col[swz(ky)] = o;
            if (kyr != ky) col[swz(kyr)] = orr;
        };
        for (int e = threadIdx.x; e < C * hq; e += blockDim.x) {
            const int c = e >> (ln2 - 1), ky = e & (hq - 1);
            item(c, ky);
            if (ky == 0) item(c, hq);
        }
        __syncthreads();
    }
    if (a.mode != COL_FWD) F = block_fft<+1>(F, G, n2, C, ld, ptw);
    cpx<T>* dst = out + (size_t)kx0 * n2;
    for (int e = threadIdx.x; e < C * n2; e += blockDim.x) dst[e] = F[(e >> ln2) * ld + swz(e & (n2 - 1))];
}

template <typename T>
__global__ void __launch_bounds__(FftBounds<T>::threads, FftBounds<T>::minb) col_pass_kernel(const cpx<T>* in, cpx<T>* out,  // may alias (in place)
                                                       int n1, int n2, int C,
                                                       const cpx<T>* __restrict__ pt2, const T* __restrict__ Kh,
                                                       ColArgs<T> a) {
    col_pass_body<T>(in, out, n1, n2, C, pt2, Kh, a, blockIdx.x, blockIdx.y);
}

// ------------------------------------------------------------------ row inverse (C2R)
// grid: n2 / R blocks.  mode ROW_PLAIN: write the real rows (+ offset).  ROW_TAU: write
// tau13 and reduce max |v0| of the celerity law into sc->vmax_bits.
enum RowMode { ROW_PLAIN = 0, ROW_TAU = 1 };

// celerity law (Sec. 3.2.3 Hamiltonian; Sec. 4.1 prescribed), parameters in the field type
template <typename T>
struct VelLaw {
    int mode;            // FDM_V_PRESCRIBED or FDM_V_STRESS
    int friction;        // tau_y != 0 and stress driven
    T v0, mobility;
    double tau_y, beta;  // lattice friction (FP64; evaluated only when friction != 0)
    const T* mfac;       // per-cell mobility factor m(x) (heterogeneous drag, Sec. 5.3), or null
};

template <typename T> VelLaw<T> make_vel(const fdm_params& p, const void* mfac = nullptr) {
    VelLaw<T> v;
    v.mfac = static_cast<const T*>(mfac);
    v.mode = p.velocity_mode;
    v.friction = (p.tau_y != 0.0 && p.velocity_mode == FDM_V_STRESS) ? 1 : 0;
    v.v0 = T(p.v0);
    v.mobility = T(p.mobility);
    v.tau_y = p.tau_y;
    v.beta = p.beta;
    return v;
}

template <typename T>
__device__ __forceinline__ T celerity(const VelLaw<T>& v, T tau, T up, double phi_ref) {
    if (v.mode == FDM_V_PRESCRIBED) return v.v0;
    if (!v.friction) return -(v.mobility * tau);
    const T fr = T(v.tau_y * cos(((double)up + phi_ref) / v.beta));
    return v.mobility * (fr - tau);
}

// dt from the CFL rule |v0|max dt / dx = CFL (Sec. 4.3, Sec. 5.2), in FP64
__device__ __forceinline__ double cfl_dt(double vmax, double cfl, double dx, double dt_max) {
    double dtd;
    if (vmax > 0.0) {
        dtd = cfl * dx / vmax;
        if (dt_max > 0.0 && dtd > dt_max) dtd = dt_max;
    } else {
        dtd = dt_max > 0.0 ? dt_max : 0.0;
    }
    return dtd;
}

template <typename T>
struct RowArgs {
    VelLaw<T> vel;
    int mode;
    const void* phi0;          // ROW_TAU: the two state buffers (U13 is needed for friction)
    const void* phi1;
    fdm_dev_scalars* sc;       // ROW_TAU: scalars of instance 0
    int gated;
    T offset;                  // ROW_PLAIN: added to every output value
    double cfl, dx, dt_max;    // ROW_TAU: time-step rule (FP64)
};

// body of one block: rows [tile R, tile R + R) of instance inst; ntiles = row blocks per
// instance (the last of them to finish computes the step's dt)
template <typename T>
__device__ __forceinline__ void row_inverse_body(const cpx<T>* spec, T* dst, int n1, int n2, int R,
                                                 const cpx<T>* __restrict__ tw1, const cpx<T>* __restrict__ pt1,
                                                 RowArgs<T> a, int tile, int inst, int ntiles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = n1 >> 1;
    const int ld = padded_len(L);
    cpx<T>* A = reinterpret_cast<cpx<T>*>(smem_raw);
    __shared__ int s_run, s_cur;
    
    if (threadIdx.x == 0) {
        InstCtl ctl{a.mode == ROW_TAU ? a.sc : nullptr, a.gated};
        inst_state(ctl, inst, &s_run, &s_cur);
    }
    __syncthreads();
    if (!s_run) return;
    cpx<T>* B = A + R * ld;   // second buffer (FP32)
    const cpx<T>* ptw = stage_twiddles<T>(pt1, A + fft_buffers<T>() * R * ld, L);
    const size_t nn = (size_t)n1 * n2;
    spec += inst * (nn / 2);
    dst += inst * nn;
    fdm_dev_scalars* sci = (a.mode == ROW_TAU) ? a.sc + inst : nullptr;
    const int y0 = tile * R;
    const int lL = 31 - __clz(L), lR = 31 - __clz(R);  // powers of two
    {
        const int total = R * L, step = blockDim.x;
        for (int e = threadIdx.x; e < total; e += step)
            copy_async(A + (e & (R - 1)) * ld + swz(e >> lR), spec + (size_t)(e >> lR) * n2 + y0 + (e & (R - 1)));
        copy_async_wait_all();
    }
    __syncthreads();
    const int hq = L >> 1;   // pairs (k, L - k), k < L/2; k = 0 also takes k = L/2
    for (int e = threadIdx.x; e < R * hq; e += blockDim.x) {
        const int r = e >> (lL - 1), k = e & (hq - 1);
        c2r_twist_pair(A + r * ld, A + r * ld, L, k, tw1);  // in place: a thread owns k and L - k
        if (k == 0) c2r_twist_pair(A + r * ld, A + r * ld, L, hq, tw1);
    }
    __syncthreads();
    const cpx<T>* z = block_fft<+1>(A, B, L, R, ld, ptw);
    T vmax = T(0);
    bool bad = false;
    unsigned long long vbits = 0ull;  // FP64: max of |v0| as magnitude bits (a NaN wins)
    const T* up = reinterpret_cast<const T*>(s_cur ? a.phi1 : a.phi0);
    if (up) up += inst * nn;
    const double phi_ref = (sci && a.vel.friction) ? sci->phi_ref : 0.0;
    const bool need_up = a.vel.friction != 0;
    for (int e = threadIdx.x; e < R * L; e += blockDim.x) {
        int r = e >> lL, m = e & (L - 1);
        cpx<T> v = z[r * ld + swz(m)];
        size_t o = (size_t)(y0 + r) * n1 + 2 * m;
        // the pair (o, o + 1) moves as one aligned vector (o is even)
        if (a.mode == ROW_TAU) {
            cpx<T> u = mk(T(0), T(0));
            if (need_up) u = *reinterpret_cast<const cpx<T>*>(up + o);
            T c0 = celerity(a.vel, v.x, u.x, phi_ref), c1 = celerity(a.vel, v.y, u.y, phi_ref);
            if (a.vel.mfac) {
                const cpx<T> mf = *reinterpret_cast<const cpx<T>*>(a.vel.mfac + inst * nn + o);
                c0 = c0 * mf.x;
                c1 = c1 * mf.y;
            }
            if constexpr (std::is_same<T, double>::value) {
                const unsigned long long m0 = ubits(c0) & kMagBits, m1 = ubits(c1) & kMagBits;
                vbits = m0 > vbits ? m0 : vbits;
                vbits = m1 > vbits ? m1 : vbits;
            } else {
                vmax = tmax(vmax, tmax(tabs(c0), tabs(c1)));
                bad |= (c0 != c0) || (c1 != c1);
            }
            *reinterpret_cast<cpx<T>*>(dst + o) = v;
        } else {
            *reinterpret_cast<cpx<T>*>(dst + o) = mk(v.x + a.offset, v.y + a.offset);
        }
    }
    if (a.mode == ROW_TAU) {
        // NaN-aware block max through the bit pattern of |v| (max is exact in any precision)
        unsigned long long bits = vbits;
        if constexpr (!std::is_same<T, double>::value) bits = bad ? 0x7ff8000000000000ull : abs_bits((double)vmax);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long other = __shfl_xor_sync(0xffffffffu, bits, o);
            bits = other > bits ? other : bits;
        }
        if ((threadIdx.x & 31) == 0) atomicMax(&sci->vmax_bits, bits);
        // the last block of the instance to finish turns max |v0| into this step's dt, once
        // (every block's maxima are in before its fenced counter increment)
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(&sci->ri_count, 1u) == (unsigned)ntiles - 1u) {
                __threadfence();
                const double vmax = __longlong_as_double((long long)atomicAdd(&sci->vmax_bits, 0ull));
                const double dtd = cfl_dt(vmax, a.cfl, a.dx, a.dt_max);
                sci->dt_next = dtd;
                sci->dt_h_next = dtd / a.dx;   // the stencil works in cell units
                sci->ri_count = 0u;
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(FftBounds<T>::threads, FftBounds<T>::minb) row_inverse_kernel(const cpx<T>* spec, T* dst,
                                                          int n1, int n2, int R,
                                                          const cpx<T>* __restrict__ tw1,
                                                          const cpx<T>* __restrict__ pt1, RowArgs<T> a) {
    row_inverse_body<T>(spec, dst, n1, n2, R, tw1, pt1, a, blockIdx.x, blockIdx.y, gridDim.x);
}

// max |v0| of the celerity law over the nodes of a single instance for a tau13 computed outside
// the step kernels (the heterogeneous static problem), then this step's dt by the last block,
// as the inverse row kernel does after its rows
template <typename T>
__global__ void celerity_dt_kernel(const T* __restrict__ tau, const T* phi0, const T* phi1, size_t n, VelLaw<T> vel,
                                   fdm_dev_scalars* sc, double cfl, double dx, double dt_max) {
    const int cur = sc->cur;
    const T* up = cur ? phi1 : phi0;
    const double phi_ref = vel.friction ? sc->phi_ref : 0.0;
    T vmax = T(0);
    bool bad = false;
    unsigned long long vbits = 0ull;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        T c = celerity(vel, tau[i], vel.friction ? up[i] : T(0), phi_ref);
        if (vel.mfac) c = c * vel.mfac[i];
        if constexpr (std::is_same<T, double>::value) {
            const unsigned long long m = ubits(c) & kMagBits;
            vbits = m > vbits ? m : vbits;
        } else {
            vmax = tmax(vmax, tabs(c));
            bad |= (c != c);
        }
    }
    unsigned long long bits = vbits;
    if constexpr (!std::is_same<T, double>::value) bits = bad ? 0x7ff8000000000000ull : abs_bits((double)vmax);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long other = __shfl_xor_sync(0xffffffffu, bits, o);
        bits = other > bits ? other : bits;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(&sc->vmax_bits, bits);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&sc->ri_count, 1u) == gridDim.x - 1) {
            __threadfence();
            const double vm = __longlong_as_double((long long)atomicAdd(&sc->vmax_bits, 0ull));
            const double dtd = cfl_dt(vm, cfl, dx, dt_max);
            sc->dt_next = dtd;
            sc->dt_h_next = dtd / dx;
            sc->ri_count = 0u;
        }
    }
}

// ------------------------------------------------------------------ KNP stencil
constexpr int TX = 32;  // stencil block width (threads along x1)

template <typename T>
struct KnpArgs {
    VelLaw<T> vel;
    const T* lo0;            // FP32: low words of the two state buffers (U13 = hi + lo)
    const T* lo1;
    T theta;
    int theta_code;          // 1 or 2 when theta is exactly that (exact scaling), else 0
    int time_level;
    fdm_dev_scalars* sc;     // scalars of instance 0
    int gated;
};

// Stencil block shapes: block (TX, ty) threads, each updating npt nodes stacked along x2,
// with a register budget that keeps minb blocks resident per SM.  Shape 0 is the default;
// the autotuner times all of them.  Every shape computes the same node values.
template <typename T> struct KnpShapes;
template <> struct KnpShapes<float> {   // nodes are updated two at a time (packed FP32)
    static constexpr int ty[kKnpShapes] = {8, 8, 16, 8}, npt[kKnpShapes] = {4, 2, 2, 4},
                         minb[kKnpShapes] = {4, 4, 1, 3};
};
template <> struct KnpShapes<double> {
    static constexpr int ty[kKnpShapes] = {8, 8, 16, 8}, npt[kKnpShapes] = {2, 1, 1, 4},
                         minb[kKnpShapes] = {2, 2, 1, 2};
};
template <> struct KnpShapes<df> {   // nodes are updated two at a time (packed FP32 pairs)
    static constexpr int ty[kKnpShapes] = {8, 8, 16, 8}, npt[kKnpShapes] = {2, 4, 2, 2},
                         minb[kKnpShapes] = {2, 2, 1, 1};
};

// grid (n1 / tx, n2 / (ty npt), instances); block (tx, ty); thread (i, j) updates the
// nodes (bx + i, by + j + k ty), k < npt
// body of one block: the tile (tbx, tby) of instance inst, ntiles tiles per instance (the
// last to start advances the clock); thread (tx_, ty_) of a tx x TY block
template <typename T, int V>
__device__ __forceinline__ void knp_step_body(const T* phi0, const T* phi1, const T* __restrict__ tau0, int n1, int n2,
                                              int npt, KnpArgs<T> a, int tbx, int tby, int inst, int ntiles, int tx_,
                                              int ty_, int tx) {
    constexpr int TY = KnpShapes<T>::ty[V];
    constexpr int NPT = KnpShapes<T>::npt[V];
    // FP32 carries the state as a pair of words, U13 = hi + lo: the node update works on
    // differences to the node's own value and adds its increment with an exact TwoSum, so
    // the state keeps ~48 bits while all arithmetic stays on the FP32 pipes
    constexpr bool kPair = std::is_same<T, float>::value;
    __shared__ T tile[TY * NPT + 4][TX + 4];
    __shared__ T tile_lo[kPair ? TY * NPT + 4 : 1][kPair ? TX + 4 : 1];
    __shared__ T s_tau[TY * NPT][TX];
    __shared__ T s_dt;
    __shared__ int s_run, s_cur;
    const int rows = TY * npt;
    const int bx = tbx * tx, by = tby * rows;
    const int tid = ty_ * tx + tx_;
    fdm_dev_scalars* sc = a.sc + inst;
    if (tid == 0) {
        InstCtl ctl{a.sc, a.gated};
        int run, cur;
        inst_state(ctl, inst, &run, &cur);
        s_run = run;
        s_cur = cur;
        if (run) {
            // dt / h of this step, set by the inverse row kernel from max |v0|; the last block
            // of this instance to read it advances the clock, flips the state buffer and clears
            // the running max (every other block has read them by then: each reads before its
            // fenced counter increment)
            s_dt = T(sc->dt_h_next);
            __threadfence();
            const unsigned int total = (unsigned)ntiles;
            if (atomicAdd(&sc->done_count, 1u) == total - 1) {
                __threadfence();
                const double vmax = __longlong_as_double((long long)sc->vmax_bits);
                const double dtd = sc->dt_next;
                sc->step += 1;
                sc->t += dtd;
                sc->dt = dtd;
                sc->max_abs_v0 = vmax;
                if (!(dtd == dtd) || !(vmax == vmax) || isinf(dtd)) sc->status = FDM_ERR_NONFINITE;
                sc->vmax_bits = 0ull;
                sc->done_count = 0u;
                sc->cur = cur ^ 1;
                if (a.gated && sc->steps_left > 0) sc->steps_left -= 1;
            }
        }
    }
    __syncthreads();
    if (!s_run) return;
    const size_t nn = (size_t)n1 * n2;
    const T* phi = (s_cur ? phi1 : phi0) + inst * nn;
    T* out = const_cast<T*>(s_cur ? phi0 : phi1) + inst * nn;
    const T* tau = tau0 + inst * nn;
    const T* lo_in = kPair ? (s_cur ? a.lo1 : a.lo0) + inst * nn : nullptr;
    T* lo_out = kPair ? const_cast<T*>(s_cur ? a.lo0 : a.lo1) + inst * nn : nullptr;
    const int x = bx + tx_;
    T tv[NPT];   // tau13 at this thread's nodes: loads issued ahead of the tile's
#pragma unroll
    for (int k = 0; k < NPT; ++k)
        if (k < npt) tv[k] = tau[(size_t)(by + ty_ + k * TY) * n1 + x];
    // the tile and its halo go straight from global to shared memory with asynchronous
    // copies, all of a thread's in flight at once (no register staging, no wait per element)
    for (int ly = ty_; ly < rows + 4; ly += TY) {
        const int gy = (by + ly - 2) & (n2 - 1);
        for (int lx = tx_; lx < tx + 4; lx += tx) {
            const int gx = (bx + lx - 2) & (n1 - 1);
            copy_async<T>(&tile[ly][lx], phi + (size_t)gy * n1 + gx);
            if constexpr (kPair) copy_async<T>(&tile_lo[ly][lx], lo_in + (size_t)gy * n1 + gx);
        }
    }
    copy_async_wait_all();
#pragma unroll
    for (int k = 0; k < NPT; ++k)
        if (k < npt) s_tau[ty_ + k * TY][tx_] = tv[k];
    __syncthreads();
    const T dt = s_dt;
    const int lx = tx_ + 2;
    const double phi_ref = a.vel.friction ? sc->phi_ref : 0.0;
    if constexpr (kPair) {
        // two nodes per pass, (x, y) and (x, y + TY), one in each lane of the packed FP32
        // arithmetic; an odd last node is paired with itself and written once
#pragma unroll 1
        for (int k = 0; k < npt; k += 2) {
            const int k2 = (k + 1 < npt) ? k + 1 : k;
            const int ya = by + ty_ + k * TY, yb = by + ty_ + k2 * TY;
            const int la = ty_ + k * TY + 2, lb = ty_ + k2 * TY + 2;
            const float ha = tile[la][lx], lo_a = tile_lo[la][lx], hb = tile[lb][lx], lo_b = tile_lo[lb][lx];
            f2 v0 = mkf2(celerity(a.vel, s_tau[la - 2][tx_], ha + lo_a, phi_ref),
                         celerity(a.vel, s_tau[lb - 2][tx_], hb + lo_b, phi_ref));
            if (a.vel.mfac)
                v0 = mkf2(v0.x * a.vel.mfac[inst * nn + (size_t)ya * n1 + x],
                          v0.y * a.vel.mfac[inst * nn + (size_t)yb * n1 + x]);
            // differences to each node's value, exact in the high words for nearby values;
            // the offset-equivariant update then returns the increments of U13
            const f2 h0 = mkf2(ha, hb), l0 = mkf2(lo_a, lo_b);
            auto g = [&](int i, int j) -> f2 {
                return (mkf2(tile[la + j][lx + i], tile[lb + j][lx + i]) - h0) +
                       (mkf2(tile_lo[la + j][lx + i], tile_lo[lb + j][lx + i]) - l0);
            };
            const f2 inc = knp_node_x2(g, v0, dt, a.theta, a.time_level);
            float s1, e1, hi, lo;
            two_sum(ha, inc.x, s1, e1);
            two_sum(s1, DF_ADD(lo_a, e1), hi, lo);
            out[(size_t)ya * n1 + x] = hi;
            lo_out[(size_t)ya * n1 + x] = lo;
            if (k2 != k) {
                two_sum(hb, inc.y, s1, e1);
                two_sum(s1, DF_ADD(lo_b, e1), hi, lo);
                out[(size_t)yb * n1 + x] = hi;
                lo_out[(size_t)yb * n1 + x] = lo;
            }
        }
    } else if constexpr (std::is_same<T, df>::value) {
        // two nodes per pass in the lanes of the packed FP32 instructions (double words), an
        // odd last node paired with itself and written once
#pragma unroll 1
        for (int k = 0; k < npt; k += 2) {
            const int k2 = (k + 1 < npt) ? k + 1 : k;
            const int ya = by + ty_ + k * TY, yb = by + ty_ + k2 * TY;
            const int la = ty_ + k * TY + 2, lb = ty_ + k2 * TY + 2;
            T va = celerity(a.vel, s_tau[la - 2][tx_], tile[la][lx], phi_ref);
            T vb = celerity(a.vel, s_tau[lb - 2][tx_], tile[lb][lx], phi_ref);
            if (a.vel.mfac) {
                va = va * a.vel.mfac[inst * nn + (size_t)ya * n1 + x];
                vb = vb * a.vel.mfac[inst * nn + (size_t)yb * n1 + x];
            }
            auto f = [&](int i, int j) -> df2 { return mkdf2(tile[la + j][lx + i], tile[lb + j][lx + i]); };
            const df2 res = knp_node_df2(f, mkdf2(va, vb), dt, a.theta, a.theta_code, a.time_level);
            out[(size_t)ya * n1 + x] = lane(res, 0);
            if (k2 != k) out[(size_t)yb * n1 + x] = lane(res, 1);
        }
    } else {
#pragma unroll 1
        for (int k = 0; k < npt; ++k) {
            const int y = by + ty_ + k * TY;
            const int ly = ty_ + k * TY + 2;
            const T tau_k = s_tau[ty_ + k * TY][tx_];
            const T up = tile[ly][lx];
            T v0 = celerity(a.vel, tau_k, up, phi_ref);
            if (a.vel.mfac) v0 = v0 * a.vel.mfac[inst * nn + (size_t)y * n1 + x];
            auto f = [&](int i, int j) -> T { return tile[ly + j][lx + i]; };
            out[(size_t)y * n1 + x] = knp_node<T>(f, v0, dt, a.theta, a.theta_code, a.time_level);
        }
    }
}

template <typename T, int V>
__global__ void __launch_bounds__(TX * KnpShapes<T>::ty[V], KnpShapes<T>::minb[V])
    knp_step_kernel(const T* phi0, const T* phi1, const T* __restrict__ tau0, int n1, int n2, int npt,
                    KnpArgs<T> a) {
    knp_step_body<T, V>(phi0, phi1, tau0, n1, n2, npt, a, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x * gridDim.y,
                        threadIdx.x, threadIdx.y, blockDim.x);
}

// ------------------------------------------------------------------ set-up / readout helpers
// Layer Green kernel (Sec. 3.1.2 + layer average, Sec. 3.2.1), with the inverse transform's
// normalisation folded in: Kh[kx][ky] = (1/(nz nh n1 n2)) sum_k3 m(xi) |chi-hat(k3)|^2,
// m = -mu (n2^2 + 2 n1^2 n3^2/(1-nu)).
// w3[k3] = |chi-hat(k3)|^2 for k3 in [0, nz/2] (host table), even in k3.
__global__ void kernel_table_kernel(double* __restrict__ Kh, int n1, int n2, int nz, int nh,
                                    double mu, double nu, const double* __restrict__ w3) {
    const int w = n2 / 2 + 1;
    const int total = (n1 / 2 + 1) * w;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        int kx = i / w, ky = i - kx * w;
        double x1 = (double)kx / (double)n1, x2 = (double)ky / (double)n2;
        double acc = 0.0;
        for (int k3 = 0; k3 <= nz / 2; ++k3) {
            double x3 = (double)k3 / (double)nz;
            double r2 = x1 * x1 + x2 * x2 + x3 * x3;
            if (r2 == 0.0) continue;
            double ir2 = 1.0 / r2;
            double m = -mu * (x2 * x2 * ir2 + 2.0 * (x1 * x1 * ir2) * (x3 * x3 * ir2) / (1.0 - nu));
            double mult = (k3 == 0 || 2 * k3 == nz) ? 1.0 : 2.0;
            acc += mult * m * w3[k3];
        }
        Kh[i] = acc / ((double)nz * (double)nh) / ((double)n1 * (double)n2);
    }
}

// One stress component of the layered eigen-distortion on a plane of the 3-D cell (Sec.
// 3.1.2), Voigt index comp (11, 22, 33, 23, 13, 12).  Closed forms of the isotropic
// Green-operator stress per unit U13-hat, n = xi/|xi|:
//   11: 2 mu n1 n3 (1 - n1^2)/(1 - nu)     22: 2 mu n1 n3 (nu - n2^2)/(1 - nu)
//   33: 2 mu n1 n3 (1 - n3^2)/(1 - nu)     23: mu n1 n2 (1 - 2 n3^2/(1 - nu))
//   13: -mu (n2^2 + 2 n1^2 n3^2/(1 - nu))  12: mu n2 n3 (1 - 2 n1^2/(1 - nu))
// Kh[kx][ky] = (1/(nz n1 n2)) sum_{k3 = 0}^{nz/2} mult m(xi1, xi2, xi3) w3[k3] at kx, ky, k3
// >= 0; w3 holds D(k3) cos or, for symbols odd in n3, D(k3) sin of 2 pi k3 (x3 - (nh - 1)/2)
// / nz (host table, zero at the x3 Nyquist index for odd symbols).  A symbol odd in n1 (n2)
// is zero at the x1 (x2) Nyquist index.
__device__ __forceinline__ double stress_symbol(int comp, double x1, double x2, double x3, double mu,
                                                double nu) {
    const double ir2 = 1.0 / (x1 * x1 + x2 * x2 + x3 * x3);
    const double q1 = x1 * x1 * ir2, q2 = x2 * x2 * ir2, q3 = x3 * x3 * ir2, inu = 1.0 / (1.0 - nu);
    switch (comp) {
        case 0: return 2.0 * mu * (x1 * x3 * ir2) * (1.0 - q1) * inu;
        case 1: return 2.0 * mu * (x1 * x3 * ir2) * (nu - q2) * inu;
        case 2: return 2.0 * mu * (x1 * x3 * ir2) * (1.0 - q3) * inu;
        case 3: return mu * (x1 * x2 * ir2) * (1.0 - 2.0 * q3 * inu);
        case 4: return -mu * (q2 + 2.0 * q1 * q3 * inu);
        default: return mu * (x2 * x3 * ir2) * (1.0 - 2.0 * q1 * inu);
    }
}

__global__ void stress_table_kernel(double* __restrict__ Kh, int n1, int n2, int nz, int comp, double mu,
                                    double nu, const double* __restrict__ w3) {
    const int w = n2 / 2 + 1;
    const int total = (n1 / 2 + 1) * w;
    const bool odd1 = comp <= 3, odd2 = comp == 3 || comp == 5;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        int kx = i / w, ky = i - kx * w;
        double acc = 0.0;
        if (!(odd1 && 2 * kx == n1) && !(odd2 && 2 * ky == n2)) {
            double x1 = (double)kx / (double)n1, x2 = (double)ky / (double)n2;
            for (int k3 = 0; k3 <= nz / 2; ++k3) {
                double x3 = (double)k3 / (double)nz;
                if (x1 == 0.0 && x2 == 0.0 && k3 == 0) continue;
                double mult = (k3 == 0 || 2 * k3 == nz) ? 1.0 : 2.0;
                acc += mult * stress_symbol(comp, x1, x2, x3, mu, nu) * w3[k3];
            }
        }
        Kh[i] = acc / (double)nz / ((double)n1 * (double)n2);
    }
}

// FP32 word pairs -> FP64 (exact: hi + lo has at most 48 significant bits)
__global__ void pair_to_double_kernel(const float* __restrict__ hi, const float* __restrict__ lo,
                                      double* __restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (double)hi[i] + (double)lo[i];
}
void launch_pair_to_double(const float* hi, const float* lo, double* out, size_t n, cudaStream_t s) {
    pair_to_double_kernel<<<4 * 152, 256, 0, s>>>(hi, lo, out, n);
}

template <typename T>
__global__ void convert_kernel(const double* __restrict__ a, T* __restrict__ b, size_t n, double offset) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] = T(a[i] - offset);
}

// curl inverse on the forward 2-D spectra (transposed, packed) of alpha11 (sa) and alpha12
// (sb): U-hat = i (a11-hat xi2 - a12-hat xi1)/|xi|^2 with odd uses zeroed at Nyquist (G8),
// normalised by 1/(n1 n2); DC = mean_up13.  Also per-block partial sums for the divergence
// residual |xi1 a11 + xi2 a12|^2 and |xi|^2 |alpha|^2 (Hermitian weights).
struct CurlArgs { double dx, mean_up13; };

__device__ __forceinline__ double xi_of(int k, int n, double dx) {
    int ks = k <= n / 2 ? k : k - n;
    return 6.283185307179586476925286766559 * (double)ks / ((double)n * dx);
}

template <typename T>
__global__ void curl_inverse_kernel(const cpx<T>* __restrict__ sa, const cpx<T>* __restrict__ sb,
                                    cpx<T>* __restrict__ out, int n1, int n2, CurlArgs c,
                                    double* __restrict__ partials) {
    __shared__ double red[32];
    const int L = n1 / 2;
    const size_t total = (size_t)L * n2;
    const double scl = 1.0 / ((double)n1 * (double)n2);
    double num = 0.0, den = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        int kx = (int)(i / n2), ky = (int)(i - (size_t)kx * n2);
        double xi2 = xi_of(ky, n2, c.dx), o2 = (2 * ky == n2) ? 0.0 : xi2;
        cpx<T> za = sa[i], zb = sb[i];
        if (kx > 0) {
            double xi1 = xi_of(kx, n1, c.dx);
            double ar = (double)za.x, ai = (double)za.y, br = (double)zb.x, bi = (double)zb.y;
            double dr = xi1 * ar + o2 * br, di = xi1 * ai + o2 * bi;
            num += 2.0 * (dr * dr + di * di);
            den += 2.0 * (xi1 * xi1 + o2 * o2) * (ar * ar + ai * ai + br * br + bi * bi);
            double q = xi1 * xi1 + xi2 * xi2;
            // w = a11 xi2(odd) - a12 xi1 ; U = i w / q
            double wr = ar * o2 - br * xi1, wi = ai * o2 - bi * xi1;
            out[i] = mk(T(-wi / q * scl), T(wr / q * scl));
        } else {
            // unpack the two real columns kx = 0 and kx = n1/2 of each field
            int kr = (n2 - ky) & (n2 - 1);
            cpx<T> za_r = conj(sa[kr]), zb_r = conj(sb[kr]);
            cpx<double> A0 = mk(0.5 * ((double)za.x + (double)za_r.x), 0.5 * ((double)za.y + (double)za_r.y));
            cpx<double> AN = mk(0.5 * ((double)za.y - (double)za_r.y), -0.5 * ((double)za.x - (double)za_r.x));
            cpx<double> B0 = mk(0.5 * ((double)zb.x + (double)zb_r.x), 0.5 * ((double)zb.y + (double)zb_r.y));
            cpx<double> BN = mk(0.5 * ((double)zb.y - (double)zb_r.y), -0.5 * ((double)zb.x - (double)zb_r.x));
            // kx = 0: xi1 = 0; kx = n1/2: xi1 odd-zeroed, even use keeps pi/dx
            double xiN = 3.14159265358979323846 / c.dx;
            {
                double dr = o2 * B0.x, di = o2 * B0.y;
                num += dr * dr + di * di;
                den += o2 * o2 * (A0.x * A0.x + A0.y * A0.y + B0.x * B0.x + B0.y * B0.y);
                dr = o2 * BN.x; di = o2 * BN.y;
                num += dr * dr + di * di;
                den += o2 * o2 * (AN.x * AN.x + AN.y * AN.y + BN.x * BN.x + BN.y * BN.y);
            }
            cpx<double> U0 = mk(0.0, 0.0), UN = mk(0.0, 0.0);
            double q0 = xi2 * xi2, qN = xiN * xiN + xi2 * xi2;
            if (q0 > 0.0) U0 = mk(-(A0.y * o2) / q0, (A0.x * o2) / q0);
            UN = mk(-(AN.y * o2) / qN, (AN.x * o2) / qN);
            // repack U0 + i UN
            cpx<double> r = mk(U0.x - UN.y, U0.y + UN.x);
            if (ky == 0) r = mk(c.mean_up13 / scl, 0.0);   // UN(0) = 0 (o2 = 0)
            out[i] = mk(T(r.x * scl), T(r.y * scl));
        }
    }
    double s1 = block_sum(num, red);
    double s2 = block_sum(den, red);
    if (threadIdx.x == 0) { partials[2 * blockIdx.x] = s1; partials[2 * blockIdx.x + 1] = s2; }
}

// info: FP64 sums over the staggered Nye components of the current state, unscaled by the
// cell size (the host divides the totals by dx once): per block, sum |d12|, sum d12,
// sum |d11|, sum d11, sum |(d11, d12)| and sum U13, with d12 = U(x+1, y) - U(x, y) = dx
// alpha12 and d11 = U(x, y+1) - U(x, y) = -dx alpha11.  The positive and negative parts of
// each component follow from (sum |d| +- sum d) / 2.  The buffer of the current state is
// chosen on the device (sc->cur; buffer 0 without scalars).
template <typename T>
__global__ void alpha_sums_kernel(const T* __restrict__ phi0, const T* __restrict__ phi1,
                                  const T* __restrict__ lo0, const T* __restrict__ lo1,
                                  const fdm_dev_scalars* __restrict__ sc, int n1, int n2,
                                  double* __restrict__ partials) {
    __shared__ double red[32];
    const int cur = sc ? sc->cur : 0;
    const T* phi = cur ? phi1 : phi0;
    const T* lo = cur ? lo1 : lo0;
    double s[6] = {0, 0, 0, 0, 0, 0};
    const size_t total = (size_t)n1 * n2;
    auto val = [&](size_t k) -> double { return lo ? (double)phi[k] + (double)lo[k] : (double)phi[k]; };
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        int y = (int)(i / n1), x = (int)(i - (size_t)y * n1);
        double u = val(i);
        double d12 = val((size_t)y * n1 + ((x + 1) & (n1 - 1))) - u;
        double d11 = val((size_t)((y + 1) & (n2 - 1)) * n1 + x) - u;
        s[0] += fabs(d12);
        s[1] += d12;
        s[2] += fabs(d11);
        s[3] += d11;
        s[4] += tsqrt(d11 * d11 + d12 * d12);
        s[5] += u;
    }
    for (int q = 0; q < 6; ++q) {
        double r = block_sum(s[q], red);
        if (threadIdx.x == 0) partials[6 * blockIdx.x + q] = r;
    }
}

// U13 of the current state as FP64 against a stored copy: per block sum (U - prev)^2 and
// sum prev^2, then prev <- U (first = 1: only the copy, partial sums zero)
template <typename T>
__global__ void state_change_kernel(const T* __restrict__ phi0, const T* __restrict__ phi1, const T* __restrict__ lo0,
                                    const T* __restrict__ lo1, const fdm_dev_scalars* __restrict__ sc, size_t n,
                                    double* __restrict__ prev, int first, double* __restrict__ partials) {
    __shared__ double red[32];
    const int cur = sc->cur;
    const double ref = sc->phi_ref;
    const T* phi = cur ? phi1 : phi0;
    const T* lo = cur ? lo1 : lo0;
    double dd = 0.0, pp = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double u = (lo ? (double)phi[i] + (double)lo[i] : (double)phi[i]) + ref;
        if (!first) {
            const double p = prev[i], d = u - p;
            dd += d * d;
            pp += p * p;
        }
        prev[i] = u;
    }
    const double r1 = block_sum(dd, red);
    const double r2 = block_sum(pp, red);
    if (threadIdx.x == 0) { partials[2 * blockIdx.x] = r1; partials[2 * blockIdx.x + 1] = r2; }
}
template <typename T>
void launch_state_change(const Dev& d, double* prev, int first, double* partials, int nblk, cudaStream_t s) {
    state_change_kernel<T><<<nblk, 256, 0, s>>>((const T*)d.phi[0], (const T*)d.phi[1], (const T*)d.phi_lo[0],
                                               (const T*)d.phi_lo[1], d.sc, (size_t)d.p.n1 * d.p.n2, prev, first,
                                               partials);
}

// velocity readout V = v0 (alpha12, -alpha11)/|alpha| (Sec. 4.1)
template <typename T>
__global__ void velocity_kernel(const T* __restrict__ a11, const T* __restrict__ a12, const T* __restrict__ tau,
                                const T* __restrict__ phi, T* __restrict__ v1, T* __restrict__ v2, size_t n,
                                VelLaw<T> p, double phi_ref) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        T c = celerity(p, tau[i], phi[i], phi_ref);
        if (p.mfac) c = c * p.mfac[i];
        T m = tsqrt(a11[i] * a11[i] + a12[i] * a12[i]);
        if (m > T(0)) { v1[i] = c * a12[i] / m; v2[i] = -c * a11[i] / m; }
        else { v1[i] = T(0); v2[i] = T(0); }
    }
}

// ------------------------------------------------------------------ launchers
constexpr size_t kMaxDynSmem = 200 * 1024;  // dynamic shared memory the FFT kernels may request

// dynamic shared memory of a transform block of nseq sequences of length L: the sequence
// buffers and the staged twiddles
template <typename T> static size_t fft_block_smem(int nseq, int L) {
    return (size_t)fft_buffers<T>() * nseq * padded_len(L) * sizeof(cpx<T>) + staged_twiddle_bytes<T>(L);
}

// R rows per row-kernel block is valid when R <= n2, R <= 16, R n1/2 <= 8 x the thread
// bound (one radix-8 butterfly per thread) and the rows fit the shared-memory limit
template <typename T> static bool row_ok(int n1, int n2, int R) {
    return R <= n2 && R <= 16 && R * (n1 / 2) <= 8 * FftBounds<T>::threads &&
           fft_block_smem<T>(R, n1 / 2) <= kMaxDynSmem;
}
template <typename T> static bool col_ok(int n1, int n2, int C) {
    return C <= n1 / 2 && C <= 16 && C * n2 <= 8 * FftBounds<T>::threads && fft_block_smem<T>(C, n2) <= kMaxDynSmem;
}

template <typename T>
int row_candidates(int n1, int n2, int* out, int max) {
    int k = 0;
    for (int R = 1; R <= 16 && k < max; R *= 2)
        if (row_ok<T>(n1, n2, R)) out[k++] = R;
    return k;
}
template <typename T>
int col_candidates(int n1, int n2, int* out, int max) {
    int k = 0;
    for (int C = 1; C <= 16 && k < max; C *= 2)
        if (col_ok<T>(n1, n2, C)) out[k++] = C;
    return k;
}

// heuristic shapes: as many valid rows as fit 40 KB of shared memory; columns until a
// block has 1024 points
template <typename T> static int pick_rows(int n1, int n2) {
    const size_t per_row = (size_t)padded_len(n1 / 2) * sizeof(cpx<T>);   // one buffer
    int R = 1;
    while (row_ok<T>(n1, n2, 2 * R) && (size_t)(2 * R) * per_row <= 40 * 1024) R *= 2;
    return R;
}
static int pick_cols(int n1, int n2) {
    int C = 1;
    while (C * n2 < 1024 && 2 * C <= n1 / 2) C *= 2;
    return C;
}

template <typename T>
LaunchGeom geometry(int n1, int n2, int R, int C, int knp_shape) {
    LaunchGeom g{};
    g.R = R > 0 ? R : pick_rows<T>(n1, n2);
    g.C = C > 0 ? C : pick_cols(n1, n2);
    g.row_smem = fft_block_smem<T>(g.R, n1 / 2);
    g.col_smem = fft_block_smem<T>(g.C, n2);
    g.row_blocks = n2 / g.R;
    g.col_blocks = (n1 / 2) / g.C;
    // the in-place FFT needs at least one thread per radix-8 butterfly; at least a warp
    g.row_threads = g.R * (n1 / 2) / 8 < 32 ? 32 : g.R * (n1 / 2) / 8;
    g.col_threads = g.C * n2 / 8 < 32 ? 32 : g.C * n2 / 8;
    g.knp_shape = (knp_shape >= 0 && knp_shape < kKnpShapes) ? knp_shape : 0;
    g.tuned = 0;
    return g;
}

template <typename T>
void knp_shape_info(int shape, int* ty, int* npt, int* minb) {
    *ty = KnpShapes<T>::ty[shape];
    *npt = KnpShapes<T>::npt[shape];
    *minb = KnpShapes<T>::minb[shape];
}

// smooth periodic U13 with kinks (|sin|) on a per-instance phase: every branch of the
// stencil is taken as on a real state
template <typename T>
__global__ void tune_fill_kernel(T* phi, int n1, int n2, int count) {
    const size_t n = (size_t)n1 * n2, total = n * count;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int inst = (int)(i / n);
        const size_t c = i - (size_t)inst * n;
        const double x = (double)(c % n1) / n1, y = (double)(c / n1) / n2;
        const double u = sinpi(2.0 * (3.0 * x + 0.1 * inst)) * cospi(4.0 * y) + 0.5 * fabs(sinpi(2.0 * (x + 2.0 * y)));
        phi[i] = T(0.05 * u);
    }
}
template <typename T>
void launch_tune_fill(const Dev& d, cudaStream_t s) {
    tune_fill_kernel<T><<<4 * 152, 256, 0, s>>>((T*)d.phi[0], d.p.n1, d.p.n2, d.count);
}

template <typename T>
cudaError_t configure_kernels() {
    // the FFT kernels live on shared memory: allow large dynamic allocations and ask for the
    // largest shared-memory carveout so that several blocks stay resident per SM
    const void* fns[3] = {(const void*)row_forward_kernel<T>, (const void*)row_inverse_kernel<T>,
                          (const void*)col_pass_kernel<T>};
    for (const void* f : fns) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxDynSmem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
void launch_row_forward(const Dev& d, const T* src0, const T* src1, cpx<T>* spec, double* partials, InstCtl ctl,
                        int count, cudaStream_t s) {
    const LaunchGeom& g = d.geom;
    dim3 grid(g.row_blocks, count);
    row_forward_kernel<T><<<grid, g.row_threads, g.row_smem, s>>>(src0, src1, spec, d.p.n1, d.p.n2, g.R,
                                                                (const cpx<T>*)d.tw1, (const cpx<T>*)d.pt1,
                                                                partials, ctl);
}

template <typename T>
ColArgs<T> col_args(const Dev& d, int mode, bool with_mean, int sym_odd2 = 0, int sym_imag = 0) {
    ColArgs<T> a;
    a.p = d.p;
    a.mode = mode;
    a.row_partials = with_mean ? d.row_partials : nullptr;
    a.nparts = d.p.n2;
    a.sc = d.sc;
    a.gated = d.gated;
    a.scl = T(1.0 / ((double)d.p.n1 * (double)d.p.n2));
    a.xi1_unit = T(6.283185307179586476925286766559 / ((double)d.p.n1 * d.p.dx));
    a.xi2_unit = T(6.283185307179586476925286766559 / ((double)d.p.n2 * d.p.dx));
    a.sym_odd2 = sym_odd2;
    a.sym_imag = sym_imag;
    return a;
}
template <typename T>
void launch_col(const Dev& d, const cpx<T>* in, cpx<T>* out, int mode, bool with_mean, int count, cudaStream_t s,
                int sym_odd2 = 0, int sym_imag = 0) {
    const LaunchGeom& g = d.geom;
    dim3 grid(g.col_blocks, count);
    col_pass_kernel<T><<<grid, g.col_threads, g.col_smem, s>>>(in, out, d.p.n1, d.p.n2, g.C, (const cpx<T>*)d.pt2,
                                                             (const T*)d.Kh,
                                                             col_args<T>(d, mode, with_mean, sym_odd2, sym_imag));
}

template <typename T>
RowArgs<T> row_args(const Dev& d, int mode, double offset) {
    RowArgs<T> a;
    a.vel = make_vel<T>(d.p, d.mfac);
    a.mode = mode;
    a.phi0 = d.phi[0];
    a.phi1 = d.phi[1];
    a.sc = d.sc;
    a.gated = d.gated;
    a.offset = T(offset);
    a.cfl = d.p.cfl;
    a.dx = d.p.dx;
    a.dt_max = d.p.dt_max;
    return a;
}
template <typename T>
void launch_row_inverse(const Dev& d, const cpx<T>* spec, T* dst, int mode, double offset, int count,
                        cudaStream_t s) {
    const LaunchGeom& g = d.geom;
    dim3 grid(g.row_blocks, count);
    row_inverse_kernel<T><<<grid, g.row_threads, g.row_smem, s>>>(spec, dst, d.p.n1, d.p.n2, g.R,
                                                                (const cpx<T>*)d.tw1, (const cpx<T>*)d.pt1,
                                                                row_args<T>(d, mode, offset));
}

template <typename T, int V>
void launch_knp_shape(const Dev& d, const KnpArgs<T>& a, cudaStream_t s) {
    constexpr int TY = KnpShapes<T>::ty[V];
    const int tx = d.p.n1 < TX ? d.p.n1 : TX;
    int npt = KnpShapes<T>::npt[V];
    while (npt > 1 && d.p.n2 < TY * npt) npt >>= 1;
    dim3 grid(d.p.n1 / tx, d.p.n2 / (TY * npt), d.count), block(tx, TY);
    knp_step_kernel<T, V><<<grid, block, 0, s>>>((const T*)d.phi[0], (const T*)d.phi[1], (const T*)d.tau,
                                                 d.p.n1, d.p.n2, npt, a);
}

template <typename T>
KnpArgs<T> knp_args(const Dev& d) {
    KnpArgs<T> a;
    a.vel = make_vel<T>(d.p, d.mfac);
    a.lo0 = (const T*)d.phi_lo[0];
    a.lo1 = (const T*)d.phi_lo[1];
    a.theta = T(d.p.theta);
    a.theta_code = d.p.theta == 1.0 ? 1 : (d.p.theta == 2.0 ? 2 : 0);
    a.time_level = d.p.time_level;
    a.sc = d.sc;
    a.gated = d.gated;
    return a;
}
template <typename T>
void launch_knp(const Dev& d, cudaStream_t s) {
    const KnpArgs<T> a = knp_args<T>(d);
    switch (d.geom.knp_shape) {
        case 1: launch_knp_shape<T, 1>(d, a, s); break;
        case 2: launch_knp_shape<T, 2>(d, a, s); break;
        case 3: launch_knp_shape<T, 3>(d, a, s); break;
        default: launch_knp_shape<T, 0>(d, a, s); break;
    }
}

// one kernel of a step for every instance of the group (Sec. 3.1.1: static solve with U^n,
// then transport); U^n is buffer sc[i].cur of instance i
template <typename T>
void launch_phase(const Dev& d, int phase, cudaStream_t s) {
    cpx<T>* spec = (cpx<T>*)d.spec;
    InstCtl ctl{d.sc, d.gated};
    switch (phase) {
        case 0: launch_row_forward<T>(d, (const T*)d.phi[0], (const T*)d.phi[1], spec, d.row_partials, ctl, d.count, s); break;
        case 1: launch_col<T>(d, spec, spec, COL_K, true, d.count, s); break;
        case 2: launch_row_inverse<T>(d, spec, (T*)d.tau, ROW_TAU, 0.0, d.count, s); break;
        default: launch_knp<T>(d, s); break;
    }
}

template <typename T>
void launch_step(const Dev& d, cudaStream_t s) {
    for (int ph = 0; ph < kKernelsPerStep; ++ph) launch_phase<T>(d, ph, s);
}

// static solve of the current state with the group's table d.Kh, written without the
// celerity reduction to dst (single instance): e.g. sigma13 on a plane of the 3-D cell when
// d.Kh holds that plane's table
template <typename T>
void launch_static_to(const Dev& d, T* dst, cudaStream_t s) {
    launch_phase<T>(d, 0, s);
    launch_phase<T>(d, 1, s);
    launch_row_inverse<T>(d, (const cpx<T>*)d.spec, dst, ROW_PLAIN, 0.0, 1, s);
}

// one stress component of the current state (single instance) with the plane table d.Kh of
// a COL_SYM symbol (parity and type as stress_table_kernel's comp): rows, column transform with
// the symbol, inverse rows, written to dst
template <typename T>
void launch_stress_to(const Dev& d, int comp, T* dst, cudaStream_t s) {
    launch_phase<T>(d, 0, s);
    cpx<T>* spec = (cpx<T>*)d.spec;
    launch_col<T>(d, spec, spec, COL_SYM, false, 1, s, comp == 3 || comp == 5, comp != 3);
    launch_row_inverse<T>(d, (const cpx<T>*)d.spec, dst, ROW_PLAIN, 0.0, 1, s);
}

// 2-D transform of one real field (single instance) for solvers outside the step: rows then
// columns, unnormalised, into the packed transposed spectrum; and back (spec is overwritten;
// dst must not alias it)
template <typename T>
void launch_fft_forward(const Dev& d, const T* src, void* spec, cudaStream_t s) {
    InstCtl none{nullptr, 0};
    launch_row_forward<T>(d, src, src, (cpx<T>*)spec, nullptr, none, 1, s);
    launch_col<T>(d, (const cpx<T>*)spec, (cpx<T>*)spec, COL_FWD, false, 1, s);
}
template <typename T>
void launch_fft_inverse(const Dev& d, void* spec, T* dst, cudaStream_t s) {
    launch_col<T>(d, (const cpx<T>*)spec, (cpx<T>*)spec, COL_INV, false, 1, s);
    launch_row_inverse<T>(d, (const cpx<T>*)spec, dst, ROW_PLAIN, 0.0, 1, s);
}

// 2-D transforms of `count` consecutive real fields of the group's grid (unnormalised): the
// row and column kernels once each over all fields
template <typename T>
void launch_fft_forward_many(const Dev& d, const T* src, void* spec, int count, cudaStream_t s) {
    Dev q = d;
    q.sc = nullptr;
    q.gated = 0;
    InstCtl none{nullptr, 0};
    launch_row_forward<T>(q, src, src, (cpx<T>*)spec, nullptr, none, count, s);
    launch_col<T>(q, (const cpx<T>*)spec, (cpx<T>*)spec, COL_FWD, false, count, s);
}
template <typename T>
void launch_fft_inverse_many(const Dev& d, void* spec, T* dst, int count, cudaStream_t s) {
    Dev q = d;
    q.sc = nullptr;
    q.gated = 0;
    q.phi[0] = q.phi[1] = nullptr;
    q.mfac = nullptr;
    launch_col<T>(q, (const cpx<T>*)spec, (cpx<T>*)spec, COL_INV, false, count, s);
    launch_row_inverse<T>(q, (const cpx<T>*)spec, dst, ROW_PLAIN, 0.0, count, s);
}

// the step's dt from d.tau (single instance): see celerity_dt_kernel
template <typename T>
void launch_celerity_dt(const Dev& d, cudaStream_t s) {
    const size_t n = (size_t)d.p.n1 * d.p.n2;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 4) blocks = 152 * 4;
    celerity_dt_kernel<T><<<blocks, 256, 0, s>>>((const T*)d.tau, (const T*)d.phi[0], (const T*)d.phi[1], n,
                                                 make_vel<T>(d.p, d.mfac), d.sc, d.p.cfl, d.p.dx, d.p.dt_max);
}

// static solve only: tau for the current state of every instance
template <typename T>
void launch_static(const Dev& d, cudaStream_t s) {
    for (int ph = 0; ph < kKernelsPerStep - 1; ++ph) launch_phase<T>(d, ph, s);
}

template <typename T>
void launch_alpha(const Dev& d, const T* phi, T* a11, T* a12, cudaStream_t s) {
    cpx<T>* spec = (cpx<T>*)d.spec;
    cpx<T>* spec2 = (cpx<T>*)d.spec2;
    InstCtl none{nullptr, 0};
    launch_row_forward<T>(d, phi, phi, spec, nullptr, none, 1, s);
    launch_col<T>(d, spec, spec2, COL_DERIV1, false, 1, s);
    launch_row_inverse<T>(d, spec2, a12, ROW_PLAIN, 0.0, 1, s);
    launch_col<T>(d, spec, spec2, COL_DERIV2N, false, 1, s);
    launch_row_inverse<T>(d, spec2, a11, ROW_PLAIN, 0.0, 1, s);
}

template <typename T>
void launch_curl_inverse(const Dev& d, const T* a11, const T* a12, T* phi_out, double mean_up13, double phi_ref,
                         double* partials, int nblk, cudaStream_t s) {
    cpx<T>* spec = (cpx<T>*)d.spec;
    cpx<T>* spec2 = (cpx<T>*)d.spec2;
    // a11 / a12 may be the state buffers; the result goes through tau (free here)
    cpx<T>* tmp = (cpx<T>*)d.tau;
    InstCtl none{nullptr, 0};
    launch_row_forward<T>(d, a11, a11, spec, nullptr, none, 1, s);
    launch_row_forward<T>(d, a12, a12, spec2, nullptr, none, 1, s);
    launch_col<T>(d, spec, spec, COL_FWD, false, 1, s);
    launch_col<T>(d, spec2, spec2, COL_FWD, false, 1, s);
    CurlArgs c;
    c.dx = d.p.dx;
    c.mean_up13 = mean_up13 - phi_ref;
    curl_inverse_kernel<T><<<nblk, 256, 0, s>>>(spec, spec2, tmp, d.p.n1, d.p.n2, c, partials);
    launch_col<T>(d, tmp, spec, COL_INV, false, 1, s);
    launch_row_inverse<T>(d, spec, phi_out, ROW_PLAIN, 0.0, 1, s);
}

// Twiddle tables, computed in FP64 from exact rational angles (sincospi takes the fraction of
// pi, so no rounded multiple of pi enters) and rounded once to the field type:
// tw[m] = exp(-2 pi i m / n) for m < n; pt = the pass tables of an L-point transform
// (pass_table_entry).  Every path that needs these tables builds them here.
template <typename T>
__global__ void twiddle_tables_kernel(cpx<T>* __restrict__ tw, int n, cpx<T>* __restrict__ pt, int L) {
    const int len = pt ? pass_table_len(L) : 0;
    const int top = n > len ? n : len;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < top; i += gridDim.x * blockDim.x) {
        double sn, cs;
        if (tw && i < n) {
            sincospi(2.0 * (double)i / (double)n, &sn, &cs);
            tw[i] = mk(T(cs), T(-sn));
        }
        if (i < len) {
            int num, den;
            pass_table_entry(L, i, &num, &den);
            sincospi(2.0 * (double)num / (double)den, &sn, &cs);
            pt[i] = mk(T(cs), T(-sn));
        }
    }
}
template <typename T> void launch_twiddle_tables(void* tw, int n, void* pt, int L, cudaStream_t s) {
    twiddle_tables_kernel<T><<<8, 256, 0, s>>>((cpx<T>*)tw, n, (cpx<T>*)pt, L);
}

// layer weights |chi-hat(k3)|^2 = sin^2(pi k3 nh / nz) / sin^2(pi k3 / nz) for k3 in
// [0, nz/2] (nh^2 at k3 = 0): the transform of the layer's indicator (Sec. 3.2.1)
__global__ void layer_weights_kernel(double* __restrict__ w3, int nz, int nh) {
    for (int k3 = blockIdx.x * blockDim.x + threadIdx.x; k3 <= nz / 2; k3 += gridDim.x * blockDim.x) {
        if (k3 == 0) {
            w3[0] = (double)nh * (double)nh;
        } else {
            const double sn = sinpi((double)k3 * (double)nh / (double)nz), sd = sinpi((double)k3 / (double)nz);
            w3[k3] = (sn * sn) / (sd * sd);
        }
    }
}
void launch_layer_weights(double* w3, int nz, int nh, cudaStream_t s) {
    layer_weights_kernel<<<8, 256, 0, s>>>(w3, nz, nh);
}

void launch_kernel_table(double* Kh, int n1, int n2, int nz, int nh, double mu, double nu, const double* w3,
                         cudaStream_t s) {
    int total = (n1 / 2 + 1) * (n2 / 2 + 1);
    int blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    kernel_table_kernel<<<blocks, 256, 0, s>>>(Kh, n1, n2, nz, nh, mu, nu, w3);
}

void launch_stress_table(double* Kh, int n1, int n2, int nz, int comp, double mu, double nu, const double* w3,
                         cudaStream_t s) {
    int total = (n1 / 2 + 1) * (n2 / 2 + 1);
    int blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    stress_table_kernel<<<blocks, 256, 0, s>>>(Kh, n1, n2, nz, comp, mu, nu, w3);
}

template <typename T>
void launch_convert(const double* a, T* b, size_t n, double offset, cudaStream_t s) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 32) blocks = 152 * 32;
    convert_kernel<T><<<blocks, 256, 0, s>>>(a, b, n, offset);
}

template <typename T>
void launch_alpha_sums(const Dev& d, int inst, double* partials, int nblk, cudaStream_t s) {
    const size_t off = (size_t)inst * d.p.n1 * d.p.n2;
    auto at = [&](void* b) -> const T* { return b ? (const T*)b + off : nullptr; };
    alpha_sums_kernel<T><<<nblk, 256, 0, s>>>(at(d.phi[0]), at(d.phi[1]), at(d.phi_lo[0]), at(d.phi_lo[1]),
                                             d.sc ? d.sc + inst : nullptr, d.p.n1, d.p.n2, partials);
}

template <typename T>
void launch_velocity(const Dev& d, const T* a11, const T* a12, const T* tau, const T* phi, T* v1, T* v2,
                     cudaStream_t s) {
    size_t n = (size_t)d.p.n1 * d.p.n2;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 32) blocks = 152 * 32;
    velocity_kernel<T><<<blocks, 256, 0, s>>>(a11, a12, tau, phi, v1, v2, n, make_vel<T>(d.p, d.mfac), d.phi_ref_host);
}

// ------------------------------------------------------------------ persistent batched step
// All phases of all groups of a mixed-precision batch in ONE cooperative launch of resident
// blocks: for each step, the four phases in order; in a phase the blocks take the tasks
// (group, instance, tile) round-robin and run the same block bodies as the separate kernels;
// a grid-wide barrier separates the phases.  Every barrier wait is bounded: a block that waits
// longer than the limit records FDM_ERR_TIMEOUT and every block then leaves the kernel.
struct PersistGroup {
    const float* phi0;
    const float* phi1;
    float* tau;
    cpx<float>* spec;
    const float* Kh;
    const cpx<float>* tw1;
    const cpx<float>* pt1;
    const cpx<float>* pt2;
    double* row_partials;
    int n1, n2, count;
    int R, C;                     // rows / columns per transform task
    int row_tiles, col_tiles;     // transform tasks per instance
    int knp_gx, knp_gy, knp_npt;  // stencil tasks per instance (gx x gy) and nodes per thread
    InstCtl ctl;
    ColArgs<float> col;
    RowArgs<float> row;
    KnpArgs<float> knp;
};

// grid barrier with a bounded wait (state in device memory, reset before each launch)
__device__ bool grid_barrier(PersistBarrier* b) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned int* gen = &b->gen;
        const unsigned int g = *gen;
        __threadfence();
        if (atomicAdd(&b->count, 1u) == (unsigned int)(gridDim.x + b->extra) - 1u) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            const long long t0 = clock64();
            volatile int* st = &b->status;
            while (*gen == g) {
                if (*st != 0 || clock64() - t0 > b->limit_cycles) {
                    atomicCAS(&b->status, 0, (int)FDM_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
        if (*(volatile int*)&b->status != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

constexpr int kPersistShape = 2;   // the FP32 stencil shape of TX x 16 threads, two nodes each

__global__ void __launch_bounds__(kPersistThreads, 1)
    persistent_step_kernel(const PersistGroup* __restrict__ groups, int ngroups, int nsteps, PersistBarrier* bar) {
    for (int step = 0; step < nsteps; ++step) {
        for (int phase = 0; phase < kKernelsPerStep; ++phase) {
            int task = blockIdx.x, base = 0;
            for (int gi = 0; gi < ngroups; ++gi) {
                const PersistGroup& G = groups[gi];
                const int per = (phase == 0 || phase == 2) ? G.row_tiles : (phase == 1 ? G.col_tiles : G.knp_gx * G.knp_gy);
                const int ntask = per * G.count;
                for (; task < base + ntask; task += gridDim.x) {
                    const int local = task - base, inst = local / per, tile = local - inst * per;
                    if (phase == 0) {
                        row_forward_body<float>(G.phi0, G.phi1, G.spec, G.n1, G.n2, G.R, G.tw1, G.pt1, G.row_partials,
                                                G.ctl, tile, inst);
                    } else if (phase == 1) {
                        col_pass_body<float>(G.spec, G.spec, G.n1, G.n2, G.C, G.pt2, G.Kh, G.col, tile, inst);
                    } else if (phase == 2) {
                        row_inverse_body<float>(G.spec, G.tau, G.n1, G.n2, G.R, G.tw1, G.pt1, G.row, tile, inst, per);
                    } else {
                        knp_step_body<float, kPersistShape>(G.phi0, G.phi1, G.tau, G.n1, G.n2, G.knp_npt, G.knp,
                                                            tile % G.knp_gx, tile / G.knp_gx, inst, per,
                                                            threadIdx.x & (TX - 1), threadIdx.x / TX, TX);
                    }
                    __syncthreads();   // the next task reuses the block's shared memory
                }
                base += ntask;
            }
            if (!grid_barrier(bar)) return;
        }
    }
}

// persistent shapes of a group: transforms with one radix-8 butterfly per thread at most
fdm_status persist_group(const Dev& d, PersistGroup* out, size_t* smem) {
    const int n1 = d.p.n1, n2 = d.p.n2, L = n1 / 2;
    if (n1 < TX || n2 < 16) return FDM_ERR_INVALID_ARG;
    int R = 16, C = 16;
    while (R > 1 && (R * L > 8 * kPersistThreads || R > n2)) R >>= 1;
    while (C > 1 && (C * n2 > 8 * kPersistThreads || C > L)) C >>= 1;
    if (R * L > 8 * kPersistThreads || C * n2 > 8 * kPersistThreads) return FDM_ERR_INVALID_ARG;
    const LaunchGeom g = geometry<float>(n1, n2, R, C);
    *smem = g.row_smem > g.col_smem ? g.row_smem : g.col_smem;
    constexpr int TY = KnpShapes<float>::ty[kPersistShape];
    int npt = KnpShapes<float>::npt[kPersistShape];
    while (npt > 1 && n2 < TY * npt) npt >>= 1;
    PersistGroup G;
    G.phi0 = (const float*)d.phi[0];
    G.phi1 = (const float*)d.phi[1];
    G.tau = (float*)d.tau;
    G.spec = (cpx<float>*)d.spec;
    G.Kh = (const float*)d.Kh;
    G.tw1 = (const cpx<float>*)d.tw1;
    G.pt1 = (const cpx<float>*)d.pt1;
    G.pt2 = (const cpx<float>*)d.pt2;
    G.row_partials = d.row_partials;
    G.n1 = n1;
    G.n2 = n2;
    G.count = d.count;
    G.R = R;
    G.C = C;
    G.row_tiles = g.row_blocks;
    G.col_tiles = g.col_blocks;
    G.knp_gx = n1 / TX;
    G.knp_gy = n2 / (TY * npt);
    G.knp_npt = npt;
    G.ctl = InstCtl{d.sc, d.gated};
    G.col = col_args<float>(d, COL_K, true);
    G.row = row_args<float>(d, ROW_TAU, 0.0);
    G.knp = knp_args<float>(d);
    *out = G;
    return FDM_OK;
}

size_t persist_group_bytes() { return sizeof(PersistGroup); }

fdm_status persist_prepare(const Dev* const* groups, int ngroups, void* host_desc, size_t* smem) {
    *smem = 0;
    PersistGroup* g = static_cast<PersistGroup*>(host_desc);
    for (int i = 0; i < ngroups; ++i) {
        if (groups[i]->p.precision != FDM_MIXED) return FDM_ERR_INVALID_ARG;
        size_t sm = 0;
        fdm_status st = persist_group(*groups[i], &g[i], &sm);
        if (st != FDM_OK) return st;
        if (sm > *smem) *smem = sm;
    }
    return FDM_OK;
}

cudaError_t persist_launch(const void* dev_desc, int ngroups, int nsteps, PersistBarrier* bar, size_t smem,
                           cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(persistent_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_step_kernel, kPersistThreads, smem)) !=
        cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const PersistGroup* gd = static_cast<const PersistGroup*>(dev_desc);
    void* args[] = {(void*)&gd, (void*)&ngroups, (void*)&nsteps, (void*)&bar};
    return cudaLaunchCooperativeKernel((const void*)persistent_step_kernel, dim3(sms * per_sm),
                                       dim3(kPersistThreads), args, smem, s);
}

// explicit instantiations
#define FDM_INST(T)                                                                                         \
    template LaunchGeom geometry<T>(int, int, int, int, int);                                               \
    template int row_candidates<T>(int, int, int*, int);                                                    \
    template int col_candidates<T>(int, int, int*, int);                                                    \
    template void knp_shape_info<T>(int, int*, int*, int*);                                                 \
    template void launch_tune_fill<T>(const Dev&, cudaStream_t);                                            \
    template cudaError_t configure_kernels<T>();                                                            \
    template void launch_step<T>(const Dev&, cudaStream_t);                                                 \
    template void launch_phase<T>(const Dev&, int, cudaStream_t);                                           \
    template void launch_static<T>(const Dev&, cudaStream_t);                                               \
    template void launch_static_to<T>(const Dev&, T*, cudaStream_t);                                        \
    template void launch_stress_to<T>(const Dev&, int, T*, cudaStream_t);                                   \
    template void launch_fft_forward<T>(const Dev&, const T*, void*, cudaStream_t);                         \
    template void launch_celerity_dt<T>(const Dev&, cudaStream_t);                                          \
    template void launch_fft_inverse<T>(const Dev&, void*, T*, cudaStream_t);                               \
    template void launch_alpha<T>(const Dev&, const T*, T*, T*, cudaStream_t);                              \
    template void launch_curl_inverse<T>(const Dev&, const T*, const T*, T*, double, double, double*, int, \
                                         cudaStream_t);                                                     \
    template void launch_convert<T>(const double*, T*, size_t, double, cudaStream_t);                       \
    template void launch_alpha_sums<T>(const Dev&, int, double*, int, cudaStream_t);                        \
    template void launch_velocity<T>(const Dev&, const T*, const T*, const T*, const T*, T*, T*,            \
                                     cudaStream_t);                                                     \
    template void launch_twiddle_tables<T>(void*, int, void*, int, cudaStream_t);                          \
    template void launch_state_change<T>(const Dev&, double*, int, double*, int, cudaStream_t);                          \
    template void launch_fft_forward_many<T>(const Dev&, const T*, void*, int, cudaStream_t);              \
    template void launch_fft_inverse_many<T>(const Dev&, void*, T*, int, cudaStream_t);
FDM_INST(double)
FDM_INST(float)
FDM_INST(df)

}  // namespace fdm
