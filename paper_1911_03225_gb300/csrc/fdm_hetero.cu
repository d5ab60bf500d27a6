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

// ---------------------------------------------------------------------------------
// Heterogeneous elasticity for a plastic layer thinner than the cell (Sec. 3.1.2,
// heterogeneous medium; the layer of Sec. 3.2.1), FP64.  The modulus field f(x1, x2) is
// uniform through the depth of the cell, so the problem is invariant along x3 and its
// Fourier modes in x3 decouple: for each k3 = 0 .. nz/2 the strain's x3-transform
// eps-hat_k3(x1, x2) (six complex components) obeys the same fixed-point iteration as the
// 3-D problem, eps-hat_k3 <- E nz delta_k3,0 - Gamma0(xi1, xi2, xi3(k3)) * tau-hat_k3, with
// tau-hat_k3 = (C - C0) : eps-hat_k3 - C : eps-hat^p_k3 and
// eps-hat^p_k3,13 = chi-hat(k3) U13 / 2, chi-hat(k3) = sum_{j < nh} exp(-2 pi i k3 j / nz).
// Each complex component is carried as two real fields (real and imaginary parts), so one
// iteration is a pointwise polarisation, 12 (nz/2 + 1) forward real 2-D transforms (the
// step's row and column kernels, one launch each over all fields), the Green operator on
// the packed spectra, the inverse transforms and the increment norms (Parseval over k3).
// ---------------------------------------------------------------------------------
namespace {

// component order of the symmetric strain: 00 11 22 12 02 01 (02 = 13 in the paper's
// indexing)
__constant__ int kHlI[6] = {0, 1, 2, 1, 0, 0};
__constant__ int kHlJ[6] = {0, 1, 2, 2, 2, 1};

struct LayerArgs {
    int n1, n2, nz, nh, M;        // M = nz/2 + 1 modes in x3
    double mu, lam, f0;           // isotropic moduli, reference factor
    double mu0, lam0;             // reference medium
    int stress_control;
    double sigma_bar13, eps_bar13;
    size_t n;                     // n1 n2
};

// chi-hat(k3) of the layer: sum_{j < nh} exp(-2 pi i k3 j / nz)
__device__ __forceinline__ void layer_chi(int k3, int nh, int nz, double* re, double* im) {
    double sr = 0.0, si = 0.0;
    for (int j = 0; j < nh; ++j) {
        double sn, cs;
        sincospi(-2.0 * (double)k3 * (double)j / (double)nz, &sn, &cs);
        sr += cs;
        si += sn;
    }
    *re = sr;
    *im = si;
}

// field index of component c (0..5), part (0 real, 1 imaginary) of mode m
__device__ __forceinline__ size_t hl_field(int m, int c, int part) { return (size_t)m * 12 + 2 * c + part; }

// tau-hat = (C - C0) : eps-hat - C : eps-hat^p, per mode and point; the state's U13
__global__ void hl_polarise_kernel(StateRef st, const double* __restrict__ f, const double* __restrict__ eps,
                                   double* __restrict__ tau, LayerArgs a) {
    const int cur = st.sc->cur;
    const size_t total = (size_t)a.M * a.n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(i / a.n);
        const size_t q = i - (size_t)m * a.n;
        const double u = state_at<double>((const double*)st.phi0, (const double*)st.phi1, nullptr, nullptr, cur, q);
        const double fq = f[q], dl = (fq - a.f0) * a.lam, dm = (fq - a.f0) * a.mu;
        double er[6], ei[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            er[c] = eps[hl_field(m, c, 0) * a.n + q];
            ei[c] = eps[hl_field(m, c, 1) * a.n + q];
        }
        const double trr = er[0] + er[1] + er[2], tri = ei[0] + ei[1] + ei[2];
        double cr, ci;
        layer_chi(m, a.nh, a.nz, &cr, &ci);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            double tr_ = 2.0 * dm * er[c] + (c < 3 ? dl * trr : 0.0);
            double ti_ = 2.0 * dm * ei[c] + (c < 3 ? dl * tri : 0.0);
            if (c == 4) {   // - C : eps^p, eps^p_13 = chi-hat U13 / 2
                tr_ -= fq * a.mu * cr * u;
                ti_ -= fq * a.mu * ci * u;
            }
            tau[hl_field(m, c, 0) * a.n + q] = tr_;
            tau[hl_field(m, c, 1) * a.n + q] = ti_;
        }
    }
}

// -Gamma0 of the reference medium applied to the complex symmetric tensor Z at the
// frequency xi (vector form: v = Z xi, w = (v - c n (n . v)) / (mu0 |xi|^2),
// Gamma0 Z = sym(xi (x) w)), with the terms odd in an axis at its Nyquist frequency removed:
// the operator is averaged over the sign flips of those axes (reading G8)
__device__ void hl_gamma(const double zr[6], const double zi[6], const double xi_in[3], const int nyq[3],
                         double mu0, double cc, double scale, double wr[6], double wi[6]) {
#pragma unroll
    for (int c = 0; c < 6; ++c) { wr[c] = 0.0; wi[c] = 0.0; }
    int na = 0;
    for (int s = 0; s < 8; ++s) {
        if (((s & 1) && !nyq[0]) || ((s & 2) && !nyq[1]) || ((s & 4) && !nyq[2])) continue;
        ++na;
        const double xi[3] = {(s & 1) ? -xi_in[0] : xi_in[0], (s & 2) ? -xi_in[1] : xi_in[1],
                              (s & 4) ? -xi_in[2] : xi_in[2]};
        const double q2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
        double Zr[3][3], Zi[3][3];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            Zr[kHlI[c]][kHlJ[c]] = Zr[kHlJ[c]][kHlI[c]] = zr[c];
            Zi[kHlI[c]][kHlJ[c]] = Zi[kHlJ[c]][kHlI[c]] = zi[c];
        }
        double vr[3], vi[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            vr[i] = Zr[i][0] * xi[0] + Zr[i][1] * xi[1] + Zr[i][2] * xi[2];
            vi[i] = Zi[i][0] * xi[0] + Zi[i][1] * xi[1] + Zi[i][2] * xi[2];
        }
        const double nvr = (xi[0] * vr[0] + xi[1] * vr[1] + xi[2] * vr[2]) / q2;
        const double nvi = (xi[0] * vi[0] + xi[1] * vi[1] + xi[2] * vi[2]) / q2;
        double w_r[3], w_i[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            w_r[i] = (vr[i] - cc * xi[i] * nvr) / (mu0 * q2);
            w_i[i] = (vi[i] - cc * xi[i] * nvi) / (mu0 * q2);
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const int i = kHlI[c], j = kHlJ[c];
            wr[c] += 0.5 * (xi[i] * w_r[j] + xi[j] * w_r[i]);
            wi[c] += 0.5 * (xi[i] * w_i[j] + xi[j] * w_i[i]);
        }
    }
    const double sc = -scale / (double)na;
#pragma unroll
    for (int c = 0; c < 6; ++c) { wr[c] *= sc; wi[c] *= sc; }
}

// the new strain transforms of the two real fields (A: real part, B: imaginary part of the
// mode) at 2-D frequency k, from their transforms A(k), B(k) (complex, six components):
// A' = G_e A + i G_o B, B' = -i G_o A + G_e B with G_e, G_o the parts of -Gamma0 even and odd
// in (xi1, xi2) at fixed xi3, i.e. from the operator at xi = (xi1, xi2, xi3) and at
// xi' = (-xi1, -xi2, xi3)
__device__ void hl_point(const cpx<double> A[6], const cpx<double> B[6], double x1, double x2, double x3,
                         const int nyq[3], double mu0, double cc, double scale, cpx<double> Ao[6], cpx<double> Bo[6]) {
    double ar[6], ai[6], br[6], bi[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) { ar[c] = A[c].x; ai[c] = A[c].y; br[c] = B[c].x; bi[c] = B[c].y; }
    const double xi[3] = {x1, x2, x3}, xim[3] = {-x1, -x2, x3};
    double gAr[6], gAi[6], hAr[6], hAi[6], gBr[6], gBi[6], hBr[6], hBi[6];
    hl_gamma(ar, ai, xi, nyq, mu0, cc, scale, gAr, gAi);    // G(xi) A
    hl_gamma(ar, ai, xim, nyq, mu0, cc, scale, hAr, hAi);   // G(xi') A
    hl_gamma(br, bi, xi, nyq, mu0, cc, scale, gBr, gBi);
    hl_gamma(br, bi, xim, nyq, mu0, cc, scale, hBr, hBi);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        // even part E = (G + G') / 2, odd part O = (G - G') / 2
        const double eAr = 0.5 * (gAr[c] + hAr[c]), eAi = 0.5 * (gAi[c] + hAi[c]);
        const double oAr = 0.5 * (gAr[c] - hAr[c]), oAi = 0.5 * (gAi[c] - hAi[c]);
        const double eBr = 0.5 * (gBr[c] + hBr[c]), eBi = 0.5 * (gBi[c] + hBi[c]);
        const double oBr = 0.5 * (gBr[c] - hBr[c]), oBi = 0.5 * (gBi[c] - hBi[c]);
        Ao[c] = mk(eAr - oBi, eAi + oBr);    // E A + i O B
        Bo[c] = mk(eBr + oAi, eBi - oAr);    // E B - i O A
    }
}

// Green operator on the packed transposed spectra of every mode, in place, normalised by
// 1/(n1 n2); the 3-D zero frequency (mode 0, k = 0) receives nz E, with E prescribed
// (strain control) or from the polarisation's mean (stress control)
__global__ void hl_green_kernel(cpx<double>* __restrict__ sp, LayerArgs a) {
    const int L = a.n1 / 2, n2 = a.n2;
    const size_t per = (size_t)L * n2;          // packed points per field
    const size_t total = (size_t)a.M * per;
    const double scale = 1.0 / (double)a.n;     // 1 / (n1 n2)
    const double cc = (a.lam0 + a.mu0) / (a.lam0 + 2.0 * a.mu0);   // n (x) n part of the acoustic tensor's inverse
    const double two_pi = 6.283185307179586476925286766559;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(i / per);
        const size_t kq = i - (size_t)m * per;
        const int kx = (int)(kq / n2), ky = (int)(kq - (size_t)kx * n2);
        const double x3 = two_pi * (double)m / (double)a.nz;
        auto at = [&](int c, int part, int kyy) -> cpx<double>& {
            return sp[hl_field(m, c, part) * per + (size_t)kx * n2 + kyy];
        };
        const int kys = ky <= n2 / 2 ? ky : ky - n2;
        const double x2 = two_pi * (double)kys / (double)n2;
        if (kx > 0) {
            cpx<double> A[6], B[6], Ao[6], Bo[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) { A[c] = at(c, 0, ky); B[c] = at(c, 1, ky); }
            const int nyq[3] = {0, 2 * ky == n2, 2 * m == a.nz};
            hl_point(A, B, two_pi * (double)kx / (double)a.n1, x2, x3, nyq, a.mu0, cc, scale, Ao, Bo);
#pragma unroll
            for (int c = 0; c < 6; ++c) { at(c, 0, ky) = Ao[c]; at(c, 1, ky) = Bo[c]; }
            continue;
        }
        // packed column: P = C0 + i CN with C0, CN the transforms of the columns kx = 0 and
        // kx = n1/2; the thread of ky <= n2/2 unpacks ky and -ky, applies the operator at the
        // four frequencies (0, +-ky), (n1/2, +-ky) and repacks both entries
        if (ky > n2 / 2) continue;
        const int kr = (n2 - ky) & (n2 - 1);
        const bool self = kr == ky;
        cpx<double> A0[2][6], AN[2][6], B0[2][6], BN[2][6];   // [0]: ky, [1]: -ky
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            for (int part = 0; part < 2; ++part) {
                const cpx<double> z = at(c, part, ky), zr = at(c, part, kr);
                // C0(ky) = (P(ky) + conj P(-ky)) / 2, CN(ky) = (P(ky) - conj P(-ky)) / (2i)
                const cpx<double> c0 = mk(0.5 * (z.x + zr.x), 0.5 * (z.y - zr.y));
                const cpx<double> cN = mk(0.5 * (z.y + zr.y), -0.5 * (z.x - zr.x));
                const cpx<double> c0r = mk(c0.x, -c0.y), cNr = mk(cN.x, -cN.y);   // the -ky entries
                if (part == 0) { A0[0][c] = c0; AN[0][c] = cN; A0[1][c] = c0r; AN[1][c] = cNr; }
                else { B0[0][c] = c0; BN[0][c] = cN; B0[1][c] = c0r; BN[1][c] = cNr; }
            }
        }
        cpx<double> A0o[2][6], ANo[2][6], B0o[2][6], BNo[2][6];
        for (int sgn = 0; sgn < 2; ++sgn) {
            const double y2 = sgn == 0 ? x2 : -x2;
            const int nyq0[3] = {0, 2 * ky == n2, 2 * m == a.nz};
            const int nyqN[3] = {1, 2 * ky == n2, 2 * m == a.nz};
            if (m == 0 && ky == 0) {
                // 3-D zero frequency: the macroscopic strain (x nz, the x3 transform's scale)
                double E[6] = {0, 0, 0, 0, 0, 0};
                if (a.stress_control) {
                    // <tau> = A0(0) / (n1 n2 nz); E = C0^-1 : (Sigma - <tau>)
                    double S[6];
                    for (int c = 0; c < 6; ++c)
                        S[c] = (c == 4 ? a.sigma_bar13 : 0.0) - A0[0][c].x / ((double)a.n * (double)a.nz);
                    const double nu0 = a.lam0 / (2.0 * (a.lam0 + a.mu0)), trs = S[0] + S[1] + S[2];
                    for (int c = 0; c < 6; ++c) E[c] = (S[c] - (c < 3 ? nu0 / (1.0 + nu0) * trs : 0.0)) / (2.0 * a.mu0);
                } else {
                    E[4] = a.eps_bar13;
                }
                for (int c = 0; c < 6; ++c) { A0o[sgn][c] = mk(E[c] * (double)a.nz, 0.0); B0o[sgn][c] = mk(0.0, 0.0); }
            } else {
                hl_point(A0[sgn], B0[sgn], 0.0, y2, x3, nyq0, a.mu0, cc, scale, A0o[sgn], B0o[sgn]);
            }
            hl_point(AN[sgn], BN[sgn], two_pi * 0.5, y2, x3, nyqN, a.mu0, cc, scale, ANo[sgn], BNo[sgn]);
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            // repack: P(ky) = C0(ky) + i CN(ky), P(-ky) = C0(-ky) + i CN(-ky)
            at(c, 0, ky) = mk(A0o[0][c].x - ANo[0][c].y, A0o[0][c].y + ANo[0][c].x);
            at(c, 1, ky) = mk(B0o[0][c].x - BNo[0][c].y, B0o[0][c].y + BNo[0][c].x);
            if (!self) {
                at(c, 0, kr) = mk(A0o[1][c].x - ANo[1][c].y, A0o[1][c].y + ANo[1][c].x);
                at(c, 1, kr) = mk(B0o[1][c].x - BNo[1][c].y, B0o[1][c].y + BNo[1][c].x);
            }
        }
    }
}

// Parseval sums over the 3-D cell of |eps_new - eps|^2 and |eps_new|^2 (Frobenius, off-diagonal
// components twice; mode weights 1 for k3 = 0 and nz/2, 2 otherwise; / nz), then eps <- eps_new
__global__ void hl_update_kernel(const double* __restrict__ enew, double* __restrict__ eps, LayerArgs a,
                                 double* __restrict__ partials) {
    __shared__ double red[32];
    double dd = 0.0, ee = 0.0;
    const size_t total = (size_t)a.M * 12 * a.n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t fidx = i / a.n;
        const int m = (int)(fidx / 12), c = (int)((fidx % 12) / 2);
        const double w = ((m == 0 || 2 * m == a.nz) ? 1.0 : 2.0) * (c < 3 ? 1.0 : 2.0);
        const double v = enew[i], d = v - eps[i];
        dd += w * d * d;
        ee += w * v * v;
        eps[i] = v;
    }
    const double r1 = hsum_block(dd, red);
    const double r2 = hsum_block(ee, red);
    if (threadIdx.x == 0) { partials[2 * blockIdx.x] = r1; partials[2 * blockIdx.x + 1] = r2; }
}

// sigma13 = 2 f mu (eps13 - eps^p13): its layer average (tau) and its value on chosen planes
__global__ void hl_stress_kernel(StateRef st, const double* __restrict__ f, const double* __restrict__ eps,
                                 LayerArgs a, double* __restrict__ tau, const int* __restrict__ planes, int nplanes,
                                 double* __restrict__ out_planes) {
    const int cur = st.sc->cur;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < a.n; q += (size_t)gridDim.x * blockDim.x) {
        const double u = state_at<double>((const double*)st.phi0, (const double*)st.phi1, nullptr, nullptr, cur, q);
        const double g = 2.0 * f[q] * a.mu;
        double acc = 0.0;
        for (int m = 0; m < a.M; ++m) {
            double cr, ci;
            layer_chi(m, a.nh, a.nz, &cr, &ci);
            const double sr = g * (eps[hl_field(m, 4, 0) * a.n + q] - 0.5 * cr * u);
            const double si = g * (eps[hl_field(m, 4, 1) * a.n + q] - 0.5 * ci * u);
            const double w = (m == 0 || 2 * m == a.nz) ? 1.0 : 2.0;
            acc += w * (sr * cr + si * ci);   // Re(sigma-hat conj(chi-hat))
        }
        tau[q] = acc / ((double)a.nz * (double)a.nh);
        for (int p = 0; p < nplanes; ++p) {
            double s = 0.0;
            for (int m = 0; m < a.M; ++m) {
                double cr, ci, sn, cs;
                layer_chi(m, a.nh, a.nz, &cr, &ci);
                sincospi(2.0 * (double)m * (double)planes[p] / (double)a.nz, &sn, &cs);
                const double sr = g * (eps[hl_field(m, 4, 0) * a.n + q] - 0.5 * cr * u);
                const double si = g * (eps[hl_field(m, 4, 1) * a.n + q] - 0.5 * ci * u);
                const double w = (m == 0 || 2 * m == a.nz) ? 1.0 : 2.0;
                s += w * (sr * cs - si * sn);   // Re(sigma-hat exp(2 pi i m x3 / nz))
            }
            out_planes[(size_t)p * a.n + q] = s / (double)a.nz;
        }
    }
}

}  // namespace

fdm_status hetero_layer_solve(const Dev& d, const double* f_dev, double f0, bool stress_control, double load,
                              double tol, int max_iter, const int* planes_dev, int nplanes, double* tau_out,
                              double* planes_out, void* const bufs[3], double* partials, int nblk, cudaStream_t s,
                              int* iterations, double* residual) {
    const int n1 = d.p.n1, n2 = d.p.n2, nz = d.p.nz, nh = d.p.nh;
    const size_t n = (size_t)n1 * n2;
    LayerArgs a;
    a.n1 = n1;
    a.n2 = n2;
    a.nz = nz;
    a.nh = nh;
    a.M = nz / 2 + 1;
    a.mu = d.p.E / (2.0 * (1.0 + d.p.nu));
    a.lam = 2.0 * a.mu * d.p.nu / (1.0 - 2.0 * d.p.nu);
    a.f0 = f0;
    a.mu0 = f0 * a.mu;
    a.lam0 = f0 * a.lam;
    a.stress_control = stress_control ? 1 : 0;
    a.sigma_bar13 = stress_control ? load : 0.0;
    a.eps_bar13 = stress_control ? 0.0 : load;
    a.n = n;
    const int count = 12 * a.M;
    double* eps = (double*)bufs[0];
    double* work = (double*)bufs[1];
    void* spec = bufs[2];
    StateRef st{d.phi[0], d.phi[1], nullptr, nullptr, d.sc};
    // scale of the eigenstrain: rms over the cell of eps^p - <eps^p> (Frobenius), from U13
    std::vector<double> u(n);
    fdm_dev_scalars sc;
    FDM_CK(cudaMemcpyAsync(&sc, d.sc, sizeof(sc), cudaMemcpyDeviceToHost, s));
    FDM_CK(cudaStreamSynchronize(s));
    FDM_CK(cudaMemcpyAsync(u.data(), d.phi[sc.cur], n * sizeof(double), cudaMemcpyDeviceToHost, s));
    FDM_CK(cudaStreamSynchronize(s));
    const double pmean = 0.5 * ((double)nh / (double)nz) * (ksum(u.data(), n) / (double)n);
    std::vector<double> sq(n);
    for (size_t q = 0; q < n; ++q) {
        const double e = 0.5 * u[q] - pmean;
        sq[q] = (double)nh * e * e + (double)(nz - nh) * pmean * pmean;
    }
    const double prms = std::sqrt(2.0 * ksum(sq.data(), n) / ((double)n * (double)nz));
    const size_t fields = (size_t)count * n;
    FDM_CK(cudaMemsetAsync(eps, 0, fields * sizeof(double), s));
    const int eblk = (int)std::min<size_t>((a.M * n + 255) / 256, 152 * 16);
    const int gblk = (int)std::min<size_t>((a.M * n / 2 + 255) / 256, 152 * 16);
    std::vector<double> buf;
    double sums[2];
    int it = 0;
    double r = 0.0;
    fdm_status e;
    while (it < max_iter) {
        ++it;
        hl_polarise_kernel<<<eblk, 256, 0, s>>>(st, f_dev, eps, work, a);
        launch_fft_forward_many<double>(d, work, spec, count, s);
        hl_green_kernel<<<gblk, 256, 0, s>>>((cpx<double>*)spec, a);
        launch_fft_inverse_many<double>(d, spec, work, count, s);
        hl_update_kernel<<<nblk, 256, 0, s>>>(work, eps, a, partials);
        FDM_CK(cudaGetLastError());
        if ((e = host_sum(partials, nblk, s, buf, sums, 2, 2))) return e;
        const double cells = (double)n * (double)nz;
        const double scale = std::max(std::sqrt(sums[1] / (double)nz / cells), prms);
        r = scale > 0.0 ? std::sqrt(sums[0] / (double)nz / cells) / scale : 0.0;
        if (!std::isfinite(r)) return FDM_ERR_NONFINITE;
        if (tol > 0.0 && r <= tol) break;
    }
    hl_stress_kernel<<<(int)std::min<size_t>((n + 255) / 256, 152 * 16), 256, 0, s>>>(st, f_dev, eps, a, tau_out,
                                                                                     planes_dev, nplanes, planes_out);
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
