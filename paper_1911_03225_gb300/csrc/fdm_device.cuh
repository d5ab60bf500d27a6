// fdm_device.cuh -- device-side building blocks of the GB300 FDM library:
// complex arithmetic, a batched shared-memory Stockham FFT (radix 4 with one radix-2
// pass for odd log2 L), the real<->half-complex twists, and the per-node
// Kurganov-Noelle-Petrova update (Sec. 3.2.2-3.2.3 of arXiv 1911.03225).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace fdm {

template <typename T> struct cpx { T x, y; };

template <typename T> __host__ __device__ __forceinline__ cpx<T> mk(T a, T b) { cpx<T> r; r.x = a; r.y = b; return r; }
template <typename T> __host__ __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T> __host__ __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T> __host__ __device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename T> __host__ __device__ __forceinline__ cpx<T> conj(cpx<T> a) { return mk(a.x, -a.y); }
template <typename T> __host__ __device__ __forceinline__ cpx<T> scale(cpx<T> a, T s) { return mk(a.x * s, a.y * s); }
// multiply by s*i, s = +-1
template <typename T> __host__ __device__ __forceinline__ cpx<T> mul_si(cpx<T> a, int s) { return s > 0 ? mk(-a.y, a.x) : mk(a.y, -a.x); }

// twiddle w^m with w = exp(sign 2 pi i / len); table holds exp(-2 pi i m / len)
template <typename T> __device__ __forceinline__ cpx<T> twiddle(const cpx<T>* __restrict__ tw, int m, int sign) {
    cpx<T> w = tw[m];
    return sign < 0 ? w : conj(w);
}

// Batched Stockham autosort FFT in shared memory (Govindaraju et al., SC'08 formulation):
// nseq sequences of length L (power of two, >= 2), sequence s at a[s * ld].  b is scratch
// of the same shape.  Unnormalised; sign -1 forward, +1 inverse.  tw: table of length
// tw_len (a multiple of L) of exp(-2 pi i m / tw_len).  Must be called by all threads of
// the block.  Returns the buffer holding the result (a or b).
template <typename T>
__device__ cpx<T>* smem_fft(cpx<T>* a, cpx<T>* b, int L, int nseq, int ld, int sign,
                            const cpx<T>* __restrict__ tw, int tw_len) {
    cpx<T>* in = a;
    cpx<T>* out = b;
    int log2L = 31 - __clz(L);
    int Ns = 1;
    if (log2L & 1) {  // one radix-2 pass (Ns = 1: no twiddles)
        const int half = L >> 1;
        const int items = nseq * half;
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            int s = it / half, j = it - s * half;
            const cpx<T>* src = in + (size_t)s * ld;
            cpx<T>* dst = out + (size_t)s * ld;
            cpx<T> v0 = src[j], v1 = src[j + half];
            dst[2 * j] = v0 + v1;
            dst[2 * j + 1] = v0 - v1;
        }
        __syncthreads();
        cpx<T>* t = in; in = out; out = t;
        Ns = 2;
    }
    const int q = L >> 2;
    while (Ns < L) {
        const int items = nseq * q;
        const int stride = tw_len / (4 * Ns);
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            int s = it / q, j = it - s * q;
            int k = j & (Ns - 1);
            const cpx<T>* src = in + (size_t)s * ld;
            cpx<T>* dst = out + (size_t)s * ld;
            cpx<T> v0 = src[j], v1 = src[j + q], v2 = src[j + 2 * q], v3 = src[j + 3 * q];
            if (Ns > 1) {
                int m = k * stride;
                v1 = cmul(v1, twiddle(tw, m, sign));
                v2 = cmul(v2, twiddle(tw, 2 * m, sign));
                v3 = cmul(v3, twiddle(tw, 3 * m, sign));
            }
            cpx<T> t0 = v0 + v2, t1 = v0 - v2, t2 = v1 + v3, t3 = mul_si(v1 - v3, sign);
            int d = (j - k) * 4 + k;  // (j / Ns) * Ns * 4 + k
            dst[d] = t0 + t2;
            dst[d + Ns] = t1 + t3;
            dst[d + 2 * Ns] = t0 - t2;
            dst[d + 3 * Ns] = t1 - t3;
        }
        __syncthreads();
        cpx<T>* t = in; in = out; out = t;
        Ns <<= 2;
    }
    return in;
}

// ---------------------------------------------------------------------------------
// Real row of n reals <-> packed half spectrum of n/2 complex: P0 = X0 + i X_{n/2},
// P_k = X_k (1 <= k < n/2), from / to the n/2-point complex FFT of z_m = x_2m + i x_2m+1.
// Z, P: one sequence each (L = n/2 entries).  W^k = exp(-2 pi i k / n) = tw_n[k].
// ---------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void r2c_twist_pair(const cpx<T>* Z, cpx<T>* P, int L, int k,
                                               const cpx<T>* __restrict__ tw_n) {
    if (k == 0) {
        cpx<T> z0 = Z[0];
        P[0] = mk(z0.x + z0.y, z0.x - z0.y);
        return;
    }
    cpx<T> A = Z[k], B = conj(Z[L - k]);
    cpx<T> E = scale(A + B, T(0.5));
    cpx<T> D = scale(A - B, T(0.5));
    cpx<T> O = mk(D.y, -D.x);          // -i (A - B) / 2
    cpx<T> WO = cmul(tw_n[k], O);
    P[k] = E + WO;
    if (2 * k != L) P[L - k] = conj(E - WO);
}

template <typename T>
__device__ __forceinline__ void c2r_twist_pair(const cpx<T>* P, cpx<T>* Z, int L, int k,
                                               const cpx<T>* __restrict__ tw_n) {
    if (k == 0) {
        cpx<T> p0 = P[0];  // (X0, X_L)
        Z[0] = mk(p0.x + p0.y, p0.x - p0.y);
        return;
    }
    cpx<T> Xk = P[k], Xc = conj(P[L - k]);
    cpx<T> E = Xk + Xc;
    cpx<T> O = cmul(Xk - Xc, conj(tw_n[k]));  // times V^k = exp(+2 pi i k / n)
    Z[k] = mk(E.x - O.y, E.y + O.x);          // E + i O
    if (2 * k != L) Z[L - k] = mk(E.x + O.y, -E.y + O.x);  // conj(E) + i conj(O)
}

// ---------------------------------------------------------------------------------
// Kurganov-Noelle-Petrova update of one node (Sec. 3.2.3 Steps 1-4; readings G1-G7).
// f(i, j): value at node offset (i along x1, j along x2), i, j in [-2, 2].
// ---------------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T minmod3(T a, T b, T c) {
    if (a > T(0) && b > T(0) && c > T(0)) return fmin(a, fmin(b, c));
    if (a < T(0) && b < T(0) && c < T(0)) return fmax(a, fmax(b, c));
    return T(0);
}

template <typename T>
struct Side {  // one-dimensional limited quadratic on the cell on one side of the node
    T D;  // first difference toward that side, signed as phi_{j+1}-phi_j or phi_j-phi_{j-1}
    T S;  // limited second difference on that cell
};

template <typename T, typename F>
__device__ __forceinline__ T knp_node(F f, T v0, T dt, T h, T theta, int time_level) {
    const T inv_h = T(1) / h;
    const T inv_h2 = inv_h * inv_h;
    const T f0 = f(0, 0);
    // Step 1: limited second differences along x1 and x2
    T dxm3 = f(-1, 0) - f(-2, 0), dxm1 = f0 - f(-1, 0), dxp1 = f(1, 0) - f0, dxp3 = f(2, 0) - f(1, 0);
    T dym3 = f(0, -1) - f(0, -2), dym1 = f0 - f(0, -1), dyp1 = f(0, 1) - f0, dyp3 = f(0, 2) - f(0, 1);
    Side<T> xs[2], ys[2];  // [0] = + side, [1] = - side
    xs[0].D = dxp1; xs[0].S = minmod3(theta * (dxp3 - dxp1), T(0.5) * (dxp3 - dxm1), theta * (dxp1 - dxm1));
    xs[1].D = dxm1; xs[1].S = minmod3(theta * (dxp1 - dxm1), T(0.5) * (dxp1 - dxm3), theta * (dxm1 - dxm3));
    ys[0].D = dyp1; ys[0].S = minmod3(theta * (dyp3 - dyp1), T(0.5) * (dyp3 - dym1), theta * (dyp1 - dym1));
    ys[1].D = dym1; ys[1].S = minmod3(theta * (dyp1 - dym1), T(0.5) * (dyp1 - dym3), theta * (dym1 - dym3));
    // one-sided derivatives at the node
    T px[2] = {(xs[0].D - T(0.5) * xs[0].S) * inv_h, (xs[1].D + T(0.5) * xs[1].S) * inv_h};
    T qy[2] = {(ys[0].D - T(0.5) * ys[0].S) * inv_h, (ys[1].D + T(0.5) * ys[1].S) * inv_h};
    // Step 2: one-sided speeds over the four pairs
    T ap = 0, am = 0, bp = 0, bm = 0;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            T p = px[s], q = qy[t];
            T r = sqrt(p * p + q * q);
            T Hp = T(0), Hq = T(0);
            if (r > T(0)) { Hp = v0 * p / r; Hq = v0 * q / r; }
            ap = fmax(ap, Hp); am = fmin(am, Hp);
            bp = fmax(bp, Hq); bm = fmin(bm, Hq);
        }
    // Step 4 weights (G1, G5)
    T wx[2], wy[2];
    if (ap - am > T(0)) { T iw = T(1) / (ap - am); wx[0] = -am * iw; wx[1] = ap * iw; }
    else { wx[0] = T(0.5); wx[1] = T(0.5); }
    if (bp - bm > T(0)) { T iw = T(1) / (bp - bm); wy[0] = -bm * iw; wy[1] = bp * iw; }
    else { wy[0] = T(0.5); wy[1] = T(0.5); }
    // Step 3: values at the four intermediate points (G2, G3)
    T acc = T(0);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int cx = (s == 0) ? 1 : -1;
        const T ddx = (s == 0 ? ap : am) * dt;
        const T Dx = xs[s].D, Sx = xs[s].S;
        const T sgx = (s == 0) ? T(-1) : T(1);  // dx (dx -+ h)
        const T X = Dx * ddx * inv_h + Sx * ddx * (ddx + sgx * h) * (T(0.5) * inv_h2);
        const T dX = Dx * inv_h + Sx * (T(2) * ddx + sgx * h) * (T(0.5) * inv_h2);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int cy = (t == 0) ? 1 : -1;
            const T ddy = (t == 0 ? bp : bm) * dt;
            const T Dy = ys[t].D, Sy = ys[t].S;
            const T sgy = (t == 0) ? T(-1) : T(1);
            const T Y = Dy * ddy * inv_h + Sy * ddy * (ddy + sgy * h) * (T(0.5) * inv_h2);
            const T dY = Dy * inv_h + Sy * (T(2) * ddy + sgy * h) * (T(0.5) * inv_h2);
            const T cross = (f(cx, cy) - f(cx, 0) - f(0, cy) + f0) * T(cx * cy) * inv_h2;
            const T val = f0 + X + Y + cross * ddx * ddy;
            T p = dX + cross * ddy;
            T q = dY + cross * ddx;
            if (time_level == 0) {
                T r = sqrt(p * p + q * q);
                T gx = T(0), gy = T(0);
                if (r > T(0)) { gx = v0 * p / r; gy = v0 * q / r; }
                T hxx = Sx * inv_h2, hyy = Sy * inv_h2;
                T np = p - T(0.5) * dt * (hxx * gx + cross * gy);
                T nq = q - T(0.5) * dt * (cross * gx + hyy * gy);
                p = np; q = nq;
            }
            const T psi = val - dt * v0 * sqrt(p * p + q * q);
            acc += wx[s] * wy[t] * psi;
        }
    }
    return acc;
}

}  // namespace fdm
