// fdm_hetero.cu -- heterogeneous elasticity for a plastic layer filling the cell (Sec. 3.1.2,
// heterogeneous medium).  With nh = nz the plastic distortion U13(x1, x2) e1 (x) e3 does not
// vary along x3 and the static problem is antiplane shear, u = u3(x1, x2) e3, in a medium
// whose shear modulus mu(x1, x2) varies: unknown g = grad u3, sigma13 = mu (g1 - U13),
// sigma23 = mu g2.  With a reference medium mu0 the polarisation is
// tau = (mu - mu0) g - mu (U13, 0), and the paper's series expansion of the solution is
// summed by the fixed-point iteration g <- G - Gamma0 * tau(g),
// Gamma0-hat(xi) = xi (x) xi / (mu0 |xi|^2) (the odd products xi1 xi2 zeroed at the Nyquist
// indices), g-hat(0) = G.  One iteration: polarisation (pointwise), two forward 2-D
// transforms, the Green operator on the pair of spectra, two inverse transforms, and the
// increment norms.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "fdm_device.cuh"
#include "fdm_host.h"

namespace fdm {

namespace {

__device__ __forceinline__ double hsum_block(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) for (int i = 0; i < nw; ++i) r += red[i];
    __syncthreads();
    return r;
}

// U13 of the current state (buffer sc->cur), without the stored reference offset
template <typename T>
__device__ __forceinline__ T state_at(const T* phi0, const T* phi1, const T* lo0, const T* lo1, int cur, size_t i) {
    const T* p = cur ? phi1 : phi0;
    const T* l = cur ? lo1 : lo0;
    return l ? p[i] + l[i] : p[i];
}

struct StateRef {
    const void *phi0, *phi1, *lo0, *lo1;
    const fdm_dev_scalars* sc;
};

// per block: sum of U and of (U - mean)^2 (pass = 0: the first, pass = 1: the second)
template <typename T>
__global__ void hetero_moments_kernel(StateRef st, size_t n, double mean, int pass, double* partials) {
    __shared__ double red[32];
    const int cur = st.sc->cur;
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double u = (double)state_at<T>((const T*)st.phi0, (const T*)st.phi1, (const T*)st.lo0,
                                             (const T*)st.lo1, cur, i);
        s += pass == 0 ? u : (u - mean) * (u - mean);
    }
    const double r = hsum_block(s, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = r;
}

// tau1 = (mu - mu0) g1 - mu U13, tau2 = (mu - mu0) g2
template <typename T>
__global__ void hetero_polarisation_kernel(StateRef st, const T* __restrict__ mu, const T* __restrict__ g1,
                                           const T* __restrict__ g2, T* __restrict__ t1, T* __restrict__ t2,
                                           size_t n, T mu0, T phi_ref) {
    const int cur = st.sc->cur;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const T u = state_at<T>((const T*)st.phi0, (const T*)st.phi1, (const T*)st.lo0, (const T*)st.lo1, cur, i) +
                    phi_ref;
        const T m = mu[i], dm = m - mu0;
        t1[i] = dm * g1[i] - m * u;
        t2[i] = dm * g2[i];
    }
}

// the Green operator's symbol in the arithmetic of the field type (FP32 fields keep FP32)
template <typename T>
using sym_t = typename std::conditional<std::is_same<T, float>::value, float, double>::type;

// Green operator without the modulus, on the quarter (kx in [0, n1/2], ky in [0, n2/2]):
// xi1^2 / |xi|^2, xi1 xi2 / |xi|^2 (the odd product zeroed at the Nyquist indices) and
// xi2^2 / |xi|^2 at ky >= 0; the sign of the odd product follows ky's.  Zero at the origin.
template <typename S>
__global__ void hetero_gamma_table_kernel(S* __restrict__ tab, int n1, int n2) {
    const int w = n2 / 2 + 1;
    const int total = (n1 / 2 + 1) * w;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int kx = i / w, ky = i - kx * w;
        const S x1 = S(6.283185307179586476925286766559) * S(kx) / S(n1);
        const S x2 = S(6.283185307179586476925286766559) * S(ky) / S(n2);
        const S o1 = (2 * kx == n1) ? S(0) : x1, o2 = (2 * ky == n2) ? S(0) : x2;
        const S q = x1 * x1 + x2 * x2;
        const S iq = q > S(0) ? S(1) / q : S(0);
        tab[3 * i] = x1 * x1 * iq;
        tab[3 * i + 1] = o1 * o2 * iq;
        tab[3 * i + 2] = x2 * x2 * iq;
    }
}

struct GammaArgs {
    int stress_control;
    double G1, G2;        // strain control: the prescribed mean of g
    double sigma_bar13;   // stress control: the prescribed mean of sigma13
    double mu0;
};

// g-hat = -Gamma0 tau-hat on the pair of packed transposed spectra (sa: tau1, sb: tau2),
// normalised by 1/(n1 n2), written to oa, ob (not in place: the packed column kx = 0 reads
// the entries ky and n2 - ky of its inputs)
template <typename T>
__global__ void hetero_gamma0_kernel(const cpx<T>* __restrict__ sa, const cpx<T>* __restrict__ sb,
                                     cpx<T>* __restrict__ oa, cpx<T>* __restrict__ ob, int n1, int n2,
                                     const sym_t<T>* __restrict__ tab, GammaArgs a) {
    using S = sym_t<T>;
    const int L = n1 / 2, w = n2 / 2 + 1;
    const size_t total = (size_t)L * n2;
    const double N = (double)n1 * (double)n2;
    const S c = S(1.0 / (N * a.mu0));   // normalisation and 1/mu0
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int kx = (int)(i / n2), ky = (int)(i - (size_t)kx * n2);
        const bool neg = ky > n2 / 2;
        const int kyf = neg ? n2 - ky : ky;
        const cpx<T> za = sa[i], zb = sb[i];
        if (kx > 0) {
            const S* t = tab + 3 * ((size_t)kx * w + kyf);
            const S t12 = neg ? -t[1] : t[1];
            const T a11 = T(t[0] * c), a12 = T(t12 * c), a22 = T(t[2] * c);
            oa[i] = mk(-(a11 * za.x + a12 * zb.x), -(a11 * za.y + a12 * zb.y));
            ob[i] = mk(-(a12 * za.x + a22 * zb.x), -(a12 * za.y + a22 * zb.y));
        } else {
            // unpack the real columns kx = 0 and kx = n1/2 of each field (z = C0 + i CN)
            const int kr = (n2 - ky) & (n2 - 1);
            const cpx<T> ar = conj(sa[kr]), br = conj(sb[kr]);
            const T h = T(0.5);
            const cpx<T> A0 = mk(h * (za.x + ar.x), h * (za.y + ar.y)), AN = mk(h * (za.y - ar.y), -(h * (za.x - ar.x)));
            const cpx<T> B0 = mk(h * (zb.x + br.x), h * (zb.y + br.y)), BN = mk(h * (zb.y - br.y), -(h * (zb.x - br.x)));
            cpx<T> g10, g20;
            if (ky == 0) {
                double G1 = a.G1, G2 = a.G2;
                if (a.stress_control) {   // <sigma> = mu0 G + <tau>
                    G1 = (a.sigma_bar13 - (double)A0.x / N) / a.mu0;
                    G2 = -((double)B0.x / N) / a.mu0;
                }
                g10 = mk(T(G1), T(0));
                g20 = mk(T(G2), T(0));
            } else {   // xi1 = 0: the x1 part of Gamma0 vanishes, the x2 part is 1/mu0
                const T c0 = T(c);
                g10 = mk(T(0), T(0));
                g20 = mk(-(c0 * B0.x), -(c0 * B0.y));
            }
            // kx = n1/2: xi1 = pi (even use), zero in the odd product
            const S* tN = tab + 3 * ((size_t)L * w + kyf);
            const T b11 = T(tN[0] * c), b22 = T(tN[2] * c);
            const cpx<T> g1N = mk(-(b11 * AN.x), -(b11 * AN.y)), g2N = mk(-(b22 * BN.x), -(b22 * BN.y));
            oa[i] = mk(g10.x - g1N.y, g10.y + g1N.x);   // repack G0 + i GN
            ob[i] = mk(g20.x - g2N.y, g20.y + g2N.x);
        }
    }
}

// increment and size of the new iterate (per block), then g <- g_new
template <typename T>
__global__ void hetero_update_kernel(const T* __restrict__ n1v, const T* __restrict__ n2v, T* __restrict__ g1,
                                     T* __restrict__ g2, size_t n, double* __restrict__ partials) {
    __shared__ double red[32];
    double dd = 0.0, gg = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const T a = n1v[i], b = n2v[i];
        const double da = (double)(a - g1[i]), db = (double)(b - g2[i]);
        const double fa = (double)a, fb = (double)b;
        dd += da * da + db * db;
        gg += fa * fa + fb * fb;
        g1[i] = a;
        g2[i] = b;
    }
    const double r1 = hsum_block(dd, red);
    const double r2 = hsum_block(gg, red);
    if (threadIdx.x == 0) { partials[2 * blockIdx.x] = r1; partials[2 * blockIdx.x + 1] = r2; }
}

// sigma13 = mu (g1 - U13), sigma23 = mu g2
template <typename T>
__global__ void hetero_stress_kernel(StateRef st, const T* __restrict__ mu, const T* __restrict__ g1,
                                     const T* __restrict__ g2, T* __restrict__ s13, T* __restrict__ s23, size_t n,
                                     T phi_ref) {
    const int cur = st.sc->cur;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const T u = state_at<T>((const T*)st.phi0, (const T*)st.phi1, (const T*)st.lo0, (const T*)st.lo1, cur, i) +
                    phi_ref;
        s13[i] = mu[i] * (g1[i] - u);
        s23[i] = mu[i] * g2[i];
    }
}

fdm_status host_sum(const double* dev, int count, cudaStream_t s, std::vector<double>& buf, double* out, int stride,
                    int nq) {
    buf.resize((size_t)count * stride);
    FDM_CK(cudaMemcpyAsync(buf.data(), dev, buf.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    FDM_CK(cudaStreamSynchronize(s));
    std::vector<double> col(count);
    for (int q = 0; q < nq; ++q) {
        for (int b = 0; b < count; ++b) col[b] = buf[(size_t)stride * b + q];
        out[q] = ksum(col.data(), col.size());
    }
    return FDM_OK;
}

}  // namespace

template <typename T>
fdm_status hetero_solve(const Dev& d, const HeteroBuffers& hb, double mu0, bool stress_control, double load,
                        double tol, int max_iter, cudaStream_t s, int* iterations, double* residual) {
    const size_t n = (size_t)d.p.n1 * d.p.n2;
    const int nblk = d.red_blocks;
    StateRef st{d.phi[0], d.phi[1], d.phi_lo[0], d.phi_lo[1], d.sc};
    const T phi_ref = T(d.phi_ref_host);
    std::vector<double> buf;
    double sums[2];
    // scale of the plastic field: rms(U13 - <U13>)
    hetero_moments_kernel<T><<<nblk, 256, 0, s>>>(st, n, 0.0, 0, d.red);
    FDM_CK(cudaGetLastError());
    fdm_status e;
    if ((e = host_sum(d.red, nblk, s, buf, sums, 1, 1))) return e;
    const double mean = sums[0] / (double)n;
    hetero_moments_kernel<T><<<nblk, 256, 0, s>>>(st, n, mean, 1, d.red);
    FDM_CK(cudaGetLastError());
    if ((e = host_sum(d.red, nblk, s, buf, sums, 1, 1))) return e;
    const double urms = std::sqrt(sums[0] / (double)n);

    FDM_CK(cudaMemsetAsync(hb.g1, 0, n * sizeof(T), s));
    FDM_CK(cudaMemsetAsync(hb.g2, 0, n * sizeof(T), s));
    GammaArgs ga;
    ga.stress_control = stress_control ? 1 : 0;
    ga.G1 = stress_control ? 0.0 : 2.0 * load;
    ga.G2 = 0.0;
    ga.sigma_bar13 = stress_control ? load : 0.0;
    ga.mu0 = mu0;
    const int eblk = (int)std::min<size_t>((n + 255) / 256, 152 * 16);
    const int sblk = (int)std::min<size_t>((n / 2 + 255) / 256, 152 * 16);
    const int nq = (d.p.n1 / 2 + 1) * (d.p.n2 / 2 + 1);
    hetero_gamma_table_kernel<sym_t<T>><<<std::min((nq + 255) / 256, 152 * 16), 256, 0, s>>>((sym_t<T>*)hb.gam,
                                                                                           d.p.n1, d.p.n2);
    int it = 0;
    double r = 0.0;
    while (it < max_iter) {
        ++it;
        hetero_polarisation_kernel<T><<<eblk, 256, 0, s>>>(st, (const T*)hb.mu, (const T*)hb.g1, (const T*)hb.g2,
                                                          (T*)hb.t1, (T*)hb.t2, n, T(mu0), phi_ref);
        launch_fft_forward<T>(d, (const T*)hb.t1, d.spec, s);
        launch_fft_forward<T>(d, (const T*)hb.t2, d.spec2, s);
        hetero_gamma0_kernel<T><<<sblk, 256, 0, s>>>((const cpx<T>*)d.spec, (const cpx<T>*)d.spec2, (cpx<T>*)hb.t1,
                                                    (cpx<T>*)hb.t2, d.p.n1, d.p.n2, (const sym_t<T>*)hb.gam, ga);
        launch_fft_inverse<T>(d, hb.t1, (T*)d.spec, s);
        launch_fft_inverse<T>(d, hb.t2, (T*)d.spec2, s);
        hetero_update_kernel<T><<<nblk, 256, 0, s>>>((const T*)d.spec, (const T*)d.spec2, (T*)hb.g1, (T*)hb.g2, n,
                                                    d.red);
        FDM_CK(cudaGetLastError());
        if ((e = host_sum(d.red, nblk, s, buf, sums, 2, 2))) return e;
        const double scale = std::max(std::sqrt(sums[1] / (double)n), urms);
        r = scale > 0.0 ? std::sqrt(sums[0] / (double)n) / scale : 0.0;
        if (!std::isfinite(r)) return FDM_ERR_NONFINITE;
        if (tol > 0.0 && r <= tol) break;
    }
    hetero_stress_kernel<T><<<eblk, 256, 0, s>>>(st, (const T*)hb.mu, (const T*)hb.g1, (const T*)hb.g2, (T*)d.tau,
                                                (T*)hb.t2, n, phi_ref);
    FDM_CK(cudaGetLastError());
    *iterations = it;
    *residual = r;
    return FDM_OK;
}

#define FDM_HETERO_INST(T)                                                                                   \
    template fdm_status hetero_solve<T>(const Dev&, const HeteroBuffers&, double, bool, double, double, int, \
                                        cudaStream_t, int*, double*);
FDM_HETERO_INST(double)
FDM_HETERO_INST(float)
FDM_HETERO_INST(df)

}  // namespace fdm
