// fdm_device.cuh -- device-side building blocks of the GB300 FDM library:
// complex arithmetic, a batched in-place shared-memory Stockham FFT (radix 8, then one
// radix-4 or radix-2 pass), the real<->half-complex twists, and the per-node
// Kurganov-Noelle-Petrova update (Sec. 3.2.2-3.2.3 of arXiv 1911.03225).
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "fdm_df.cuh"

namespace fdm {

// aligned to its size, so that a complex value moves in one 64-bit (FP32) or 128-bit (FP64,
// double-word) access
template <typename T> struct alignas(2 * sizeof(T)) cpx { T x, y; };

template <typename T> __host__ __device__ __forceinline__ cpx<T> mk(T a, T b) { cpx<T> r; r.x = a; r.y = b; return r; }
template <typename T> __host__ __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T> __host__ __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T> __host__ __device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename T> __host__ __device__ __forceinline__ cpx<T> conj(cpx<T> a) { return mk(a.x, -a.y); }
template <typename T> __host__ __device__ __forceinline__ cpx<T> scale(cpx<T> a, T s) { return mk(a.x * s, a.y * s); }
// multiply by S i, S = +-1 (a compile-time direction: no arithmetic)
template <int S, typename T> __host__ __device__ __forceinline__ cpx<T> mul_si(cpx<T> a) {
    return S > 0 ? mk(-a.y, a.x) : mk(a.y, -a.x);
}

// twiddle w^m with w = exp(S 2 pi i / len); table holds exp(-2 pi i m / len)
template <int S, typename T> __device__ __forceinline__ cpx<T> twiddle(const cpx<T>* __restrict__ tw, int m) {
    const cpx<T> w = tw[m];
    return S < 0 ? w : conj(w);
}

// In-register DFT of R = 2, 4 or 8 points, S = -1 forward / +1 inverse, natural order.  The
// direction is a template parameter so that the rotations by W8 are additions, sign flips
// and one multiply by 1/sqrt(2), never multiplications by +-1.
template <typename T, int R> struct Dft;
template <typename T> struct Dft<T, 2> {
    template <int S> static __device__ __forceinline__ void run(cpx<T>* v) {
        cpx<T> a = v[0], b = v[1];
        v[0] = a + b; v[1] = a - b;
    }
};
template <typename T> struct Dft<T, 4> {
    template <int S> static __device__ __forceinline__ void run(cpx<T>* v) {
        cpx<T> t0 = v[0] + v[2], t1 = v[0] - v[2], t2 = v[1] + v[3], t3 = mul_si<S>(v[1] - v[3]);
        v[0] = t0 + t2; v[1] = t1 + t3; v[2] = t0 - t2; v[3] = t1 - t3;
    }
};
template <typename T> struct Dft<T, 8> {
    // radix-2 decimation in frequency, three stages, bit-reversed result reordered
    template <int S> static __device__ __forceinline__ void run(cpx<T>* a) {
        const T r = T(0.70710678118654752440084436210485);
        cpx<T> b0 = a[0] + a[4], b4 = a[0] - a[4];
        cpx<T> b1 = a[1] + a[5], b5 = a[1] - a[5];
        cpx<T> b2 = a[2] + a[6], b6 = a[2] - a[6];
        cpx<T> b3 = a[3] + a[7], b7 = a[3] - a[7];
        // b5 *= W8, b6 *= W8^2 = S i, b7 *= W8^3   (W8 = exp(S 2 pi i / 8) = (1 + S i) / sqrt 2)
        if (S < 0) {
            b5 = mk(r * (b5.x + b5.y), r * (b5.y - b5.x));
            b7 = mk(r * (b7.y - b7.x), -(r * (b7.y + b7.x)));
        } else {
            b5 = mk(r * (b5.x - b5.y), r * (b5.y + b5.x));
            b7 = mk(-(r * (b7.x + b7.y)), r * (b7.x - b7.y));
        }
        b6 = mul_si<S>(b6);
        cpx<T> c0 = b0 + b2, c2 = b0 - b2, c1 = b1 + b3, c3 = mul_si<S>(b1 - b3);
        cpx<T> c4 = b4 + b6, c6 = b4 - b6, c5 = b5 + b7, c7 = mul_si<S>(b5 - b7);
        a[0] = c0 + c1; a[4] = c0 - c1;
        a[2] = c2 + c3; a[6] = c2 - c3;
        a[1] = c4 + c5; a[5] = c4 - c5;
        a[3] = c6 + c7; a[7] = c6 - c7;
    }
};

// Shared-memory position of element i of a sequence: the low 4 index bits are XORed with
// bits 4..7, a permutation inside each aligned group of 16 that makes both the unit-stride
// reads and the strided writes of every Stockham pass touch distinct banks.
__host__ __device__ __forceinline__ int swz(int i) { return i ^ ((i >> 4) & 15); }
// sequence stride for L elements (one extra slot so that rows start on different banks)
__host__ __device__ __forceinline__ int padded_len(int L) { return L + 1; }

// Pass plan of an L-point transform (L a power of two): radix 8 while Ns * 8 <= L, then one
// radix-4 or radix-2 pass.  pass_radix(L, Ns) is the radix of the pass at sub-length Ns, 0
// once the transform is complete.  The transform, its twiddle-table length and the tables'
// contents all follow this one function.
__host__ __device__ __forceinline__ int pass_radix(int L, int Ns) {
    return Ns * 8 <= L ? 8 : (Ns * 4 == L ? 4 : (Ns * 2 == L ? 2 : 0));
}

// Twiddles of the in-place FFT, one table per pass: for the pass of radix R at sub-length Ns,
// entry (r - 1) * Ns + k holds exp(-2 pi i r k / (Ns R)), r = 1..R-1, k < Ns, so that a warp
// reads consecutive k.  pass_table_len(L) = total entries for all passes of an L-point
// transform.
__host__ __device__ __forceinline__ int pass_table_len(int L) {
    int n = 0;
    for (int Ns = 1, R; (R = pass_radix(L, Ns)) != 0; Ns *= R) n += (R - 1) * Ns;
    return n;
}
// Entry i < pass_table_len(L) of those tables is exp(-2 pi i num / den).
__host__ __device__ __forceinline__ void pass_table_entry(int L, int i, int* num, int* den) {
    int Ns = 1, R = pass_radix(L, 1);
    while (i >= (R - 1) * Ns) {
        i -= (R - 1) * Ns;
        Ns *= R;
        R = pass_radix(L, Ns);
    }
    *num = (i / Ns + 1) * (i % Ns);
    *den = Ns * R;
}

// Batched in-place FFT in shared memory: Stockham autosort passes (Govindaraju et al., SC'08)
// of radix R over nseq sequences of length L.  For j in [0, L/R), k = j mod Ns:
//   v_r = a[j + r L/R] w^(r k),  w = exp(sign 2 pi i / (Ns R)),  v = DFT_R(v),
//   a[(j - k) R + k + r Ns] = v_r.
// Each thread keeps its butterflies' values in registers between the read and the write of a
// pass (a barrier in between), so one shared buffer suffices and twice as many blocks fit
// on an SM as with a ping-pong pair (the FP64 transforms).  The FP32 transforms, whose
// blocks are limited by registers before shared memory, pass between two buffers instead
// (smem_fft_pp: one barrier per pass, the same arithmetic).  Unnormalised; sign -1
// forward, +1 inverse.
// Requires blockDim.x * 8 >= nseq * L: a thread owns at most one radix-8 butterfly per pass
// (two radix-4 or four radix-2 butterflies in the last pass).  Element i of sequence s at
// a[s * ld + swz(i)].  pt: the pass twiddle tables (pass_table_len(L) entries).  Must be
// called by all threads of the block.
template <typename T, int R, int PER, int S>
__device__ __forceinline__ void stockham_pass_ip(cpx<T>* a, int L, int nseq, int ld, int Ns,
                                                 const cpx<T>* __restrict__ ptw) {
    const int q = L / R;
    const int lq = 31 - __clz(q);
    const int items = nseq * q;
    cpx<T> v[PER][R];
    int base[PER], d[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int it = threadIdx.x + u * blockDim.x;
        if (it >= items) continue;
        const int s = it >> lq, j = it & (q - 1);
        const int k = j & (Ns - 1);
        base[u] = s * ld;
        d[u] = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) v[u][r] = a[base[u] + swz(j + r * q)];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[u][r] = cmul(v[u][r], twiddle<S>(ptw, (r - 1) * Ns + k));
        }
        Dft<T, R>::template run<S>(v[u]);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        if (threadIdx.x + u * blockDim.x >= items) continue;
#pragma unroll
        for (int r = 0; r < R; ++r) a[base[u] + swz(d[u] + r * Ns)] = v[u][r];
    }
    __syncthreads();
}

// One Stockham pass from src to a second buffer dst (the same layout): with the read and the
// write in different buffers the pass needs one barrier instead of two.
template <typename T, int R, int PER, int S>
__device__ __forceinline__ void stockham_pass_pp(const cpx<T>* src, cpx<T>* dst, int L, int nseq, int ld, int Ns,
                                                 const cpx<T>* __restrict__ ptw) {
    const int q = L / R;
    const int lq = 31 - __clz(q);
    const int items = nseq * q;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int it = threadIdx.x + u * blockDim.x;
        if (it >= items) continue;
        const int s = it >> lq, j = it & (q - 1);
        const int k = j & (Ns - 1);
        const int base = s * ld, d = (j - k) * R + k;
        cpx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[base + swz(j + r * q)];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], twiddle<S>(ptw, (r - 1) * Ns + k));
        }
        Dft<T, R>::template run<S>(v);
#pragma unroll
        for (int r = 0; r < R; ++r) dst[base + swz(d + r * Ns)] = v[r];
    }
    __syncthreads();
}

// The transform through two buffers a and b (each nseq sequences of stride ld), starting in a;
// returns the buffer that holds the result.  Same arithmetic as smem_fft_ip.
template <int S, typename T>
__device__ cpx<T>* smem_fft_pp(cpx<T>* a, cpx<T>* b, int L, int nseq, int ld, const cpx<T>* __restrict__ pt) {
    int Ns = 1;
    cpx<T>* src = a;
    cpx<T>* dst = b;
    while (pass_radix(L, Ns) == 8) {
        stockham_pass_pp<T, 8, 1, S>(src, dst, L, nseq, ld, Ns, pt);
        pt += 7 * Ns;
        Ns *= 8;
        cpx<T>* t = src; src = dst; dst = t;
    }
    const int R = pass_radix(L, Ns);
    if (R == 4) { stockham_pass_pp<T, 4, 2, S>(src, dst, L, nseq, ld, Ns, pt); return dst; }
    if (R == 2) { stockham_pass_pp<T, 2, 4, S>(src, dst, L, nseq, ld, Ns, pt); return dst; }
    return src;
}

template <int S, typename T>
__device__ void smem_fft_ip(cpx<T>* a, int L, int nseq, int ld, const cpx<T>* __restrict__ pt) {
    int Ns = 1;
    while (pass_radix(L, Ns) == 8) {
        stockham_pass_ip<T, 8, 1, S>(a, L, nseq, ld, Ns, pt);
        pt += 7 * Ns;
        Ns *= 8;
    }
    const int R = pass_radix(L, Ns);
    if (R == 4) stockham_pass_ip<T, 4, 2, S>(a, L, nseq, ld, Ns, pt);
    else if (R == 2) stockham_pass_ip<T, 2, 4, S>(a, L, nseq, ld, Ns, pt);
}

// ---------------------------------------------------------------------------------
// Real row of n reals <-> packed half spectrum of n/2 complex: P0 = X0 + i X_{n/2},
// P_k = X_k (1 <= k < n/2), from / to the n/2-point complex FFT of z_m = x_2m + i x_2m+1.
// Z, P: one padded sequence each (L = n/2 entries).  W^k = exp(-2 pi i k / n) = tw_n[k].
// ---------------------------------------------------------------------------------
// exact halves (the FP64 ones on the integer pipe, defined below)
__device__ __forceinline__ float thalf(float x);
__device__ __forceinline__ double thalf(double x);
template <typename T> __device__ __forceinline__ cpx<T> chalf(cpx<T> a) { return mk(thalf(a.x), thalf(a.y)); }

template <typename T>
__device__ __forceinline__ void r2c_twist_pair(const cpx<T>* Z, cpx<T>* P, int L, int k,
                                               const cpx<T>* __restrict__ tw_n) {
    if (k == 0) {
        cpx<T> z0 = Z[0];
        P[0] = mk(z0.x + z0.y, z0.x - z0.y);
        return;
    }
    cpx<T> A = Z[swz(k)], B = conj(Z[swz(L - k)]);
    cpx<T> E = chalf(A + B);
    cpx<T> D = chalf(A - B);
    cpx<T> O = mk(D.y, -D.x);          // -i (A - B) / 2
    cpx<T> WO = cmul(tw_n[k], O);
    P[swz(k)] = E + WO;
    if (2 * k != L) P[swz(L - k)] = conj(E - WO);
}

template <typename T>
__device__ __forceinline__ void c2r_twist_pair(const cpx<T>* P, cpx<T>* Z, int L, int k,
                                               const cpx<T>* __restrict__ tw_n) {
    if (k == 0) {
        cpx<T> p0 = P[0];  // (X0, X_L)
        Z[0] = mk(p0.x + p0.y, p0.x - p0.y);
        return;
    }
    cpx<T> Xk = P[swz(k)], Xc = conj(P[swz(L - k)]);
    cpx<T> E = Xk + Xc;
    cpx<T> O = cmul(Xk - Xc, conj(tw_n[k]));  // times V^k = exp(+2 pi i k / n)
    Z[swz(k)] = mk(E.x - O.y, E.y + O.x);          // E + i O
    if (2 * k != L) Z[swz(L - k)] = mk(E.x + O.y, -E.y + O.x);  // conj(E) + i conj(O)
}

// ---------------------------------------------------------------------------------
// Precision-typed math.  FP32 (mixed mode) keeps every operation on the FP32 pipes and
// uses the approximate special-function unit; FP64 takes its decisions, exact scalings,
// reciprocals and reciprocal square roots off the FP64 pipe (below) and keeps that pipe
// for the scheme's own additions and products.  Nothing in a float instantiation may
// promote to double: the FP64 pipe of GB300 runs at 1/64 of the FP32 rate.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ float tmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double tmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double tmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float tabs(float a) { return fabsf(a); }
__device__ __forceinline__ double tabs(double a) { return fabs(a); }
// 1/sqrt(x) for x > 0
__device__ __forceinline__ float trsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double trsqrt(double x);   // on the FP32 and integer pipes, below
// 1/x for x != 0
__device__ __forceinline__ float trcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double trcp(double x);   // on the FP32 and integer pipes, below
// x / 2 (exact)
__device__ __forceinline__ float thalf(float x) { return 0.5f * x; }
__device__ __forceinline__ double thalf(double x);
// x > 0 (false for zero and NaN)
template <typename T> __device__ __forceinline__ bool tpos(T x) { return x > T(0); }

// ---------------------------------------------------------------------------------
// Decisions on doubles, and their exact scalings by 2, made on their bit patterns.  GB300's
// FP64 pipe retires 2 lanes per SM per clock against 64 for the integer pipe, and
// comparisons, min/max, sign tests and multiplications by 1/2 or 2 occupy it like an FMA,
// so the FP64 path takes them on integers (bit for bit the same results).  With the sign bit
// cleared, the bits of a double order like its magnitude (NaN above infinity).
// ---------------------------------------------------------------------------------
constexpr unsigned long long kMagBits = 0x7fffffffffffffffull, kInfBits = 0x7ff0000000000000ull;
__device__ __forceinline__ unsigned long long ubits(double x) { return (unsigned long long)__double_as_longlong(x); }
// nonzero magnitude up to infinity: x is neither +-0 nor NaN
__device__ __forceinline__ bool mag_ok(unsigned long long m) { return m - 1ull < kInfBits; }
__device__ __forceinline__ bool tpos(double x) { return mag_ok(ubits(x)); }   // bits in [1, +inf]

__device__ __forceinline__ double dbits(unsigned long long v) { return __longlong_as_double((long long)v); }
// x / 2 exactly, on the integer pipe: one less in the exponent field for normal x above the
// least normal exponent; zero, subnormals and the least normal exponent halve their
// magnitude bits (ties to even, as the rounded product); infinities and NaN unchanged
__device__ __forceinline__ double thalf(double x) {
    const int hi = __double2hiint(x), lo = __double2loint(x);
    const unsigned e = ((unsigned)hi >> 20) & 0x7ffu;
    if (__builtin_expect(e - 2u < 0x7fdu, 1)) return __hiloint2double(hi - 0x100000, lo);
    if (e == 0x7ffu) return x;
    const unsigned long long u = ubits(x), m = u & kMagBits;
    return __longlong_as_double((long long)((u & ~kMagBits) | ((m >> 1) + (m & (m >> 1) & 1ull))));
}
// 2 x exactly, on the integer pipe: one more in the exponent field for normal x below the
// largest exponent; zero and subnormals double their magnitude bits (exact, and carries
// into the exponent field where the result is normal); the largest exponent (overflow to
// infinity), infinities and NaN through the rounded sum
__device__ __forceinline__ double ttwice(double x) {
    const int hi = __double2hiint(x), lo = __double2loint(x);
    const unsigned e = ((unsigned)hi >> 20) & 0x7ffu;
    if (__builtin_expect(e - 1u < 0x7fdu, 1)) return __hiloint2double(hi + 0x100000, lo);
    if (e != 0u) return x + x;
    const unsigned long long u = ubits(x);
    return __longlong_as_double((long long)((u & ~kMagBits) | ((u & kMagBits) << 1)));
}

// 1/sqrt(x) of a double x > 0 with no FP64 instruction: on GB300 the FP64 pipe bounds the
// FP64 stencil while the FP32 and integer pipes idle.  Newton-Raphson iteration for x^(-1/2)
// (y <- y + y (1 - x y^2) / 2) from the single-precision special-function seed, with the
// residuals formed from exact products (FMA TwoProd) and compensated sums (TwoSum) of FP32
// numbers (the error-free transformations of Dekker and Knuth), every operation an explicitly
// rounded intrinsic so that no product is contracted into a sum.  x = m 2^(2k), m in [1, 4),
// is split exactly into three floats a + b + c (24 + 24 + 5 mantissa bits); the seed y0 has
// relative error below 2^-21, the first step brings it below 2^-42 (residual to float
// accuracy), the second below 2^-84 (residual to about 2^-60 absolute); y0 + d1 + d2 is summed
// exactly in 62-bit fixed point and rounded once to the nearest double.  Relative error
// within one unit in the last place (checked against exact rational arithmetic on 4000
// values from subnormal to the largest double).  +inf gives 0, NaN gives NaN.
__device__ __forceinline__ long long fix62(float v) {   // v 2^62 truncated toward zero, |v| < 2
    const unsigned vb = __float_as_uint(v);
    const int ev = (int)((vb >> 23) & 0xffu);
    if (ev == 0) return 0;                                 // zero (or below 2^-126: < 2^-64)
    const long long m = (long long)((vb & 0x7fffffu) | 0x800000u);
    const int sh = ev - 88;                                // v = m 2^(ev - 150)
    const long long r = sh >= 0 ? (m << sh) : (sh > -40 ? (m >> -sh) : 0ll);
    return (vb >> 31) ? -r : r;
}
__device__ __forceinline__ void two_prod_rn(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}
__device__ __forceinline__ void two_sum_rn(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ double trsqrt(double x) {
    const unsigned long long u = ubits(x);
    const int e = (int)(u >> 52) & 0x7ff;
    const unsigned long long mant = u & 0xfffffffffffffull;
    if (e == 0x7ff) return mant ? x : 0.0;
    unsigned long long M;
    int E;
    if (e == 0) {                                          // subnormal: normalise the mantissa
        const int lz = __clzll((long long)mant) - 11;
        M = mant << lz;
        E = -1022 - lz;
    } else {
        M = mant | (1ull << 52);
        E = e - 1023;
    }
    const int k = E >> 1, s = E - 2 * k;                   // x = M 2^(E - 52), E = 2k + s
    const unsigned A = (unsigned)(M >> 29), B = (unsigned)(M >> 5) & 0xffffffu, Cc = (unsigned)M & 31u;
    const float a = __uint_as_float(((unsigned)(127 + s) << 23) | (A & 0x7fffffu));   // in [1, 4)
    const float b = __fmul_rn(__uint2float_rn(B), s ? 0x1p-46f : 0x1p-47f);            // exact
    const float c = __fmul_rn(__uint2float_rn(Cc), s ? 0x1p-51f : 0x1p-52f);           // exact
    const float y0 = rsqrtf(a);
    // first step: e1 = 1 - m y0^2 to float accuracy of its small terms
    float p, pe, t1, t1e;
    two_prod_rn(y0, y0, p, pe);
    two_prod_rn(a, p, t1, t1e);
    const float one_t1 = __fsub_rn(1.0f, t1);              // exact (t1 within 2^-20 of 1)
    const float e1 = __fsub_rn(one_t1, __fadd_rn(__fadd_rn(t1e, __fmul_rn(a, pe)),
                                                  __fadd_rn(__fmul_rn(b, p), __fmul_rn(c, p))));
    const float hy0 = __fmul_rn(0.5f, y0);
    const float d1 = __fmul_rn(hy0, e1);
    // second step: e2 = 1 - m (y0 + d1)^2 to about 2^-60
    float q1, q1e, q2, q2e, r, re, g, ge;
    two_prod_rn(a, pe, q1, q1e);
    two_prod_rn(b, p, q2, q2e);
    two_prod_rn(a, y0, r, re);
    const float d1x2 = __fmul_rn(2.0f, d1);
    two_prod_rn(d1x2, r, g, ge);
    float small = __fadd_rn(__fadd_rn(__fadd_rn(q1e, q2e), __fadd_rn(__fmul_rn(b, pe), __fmul_rn(c, p))),
                            __fmul_rn(d1x2, __fadd_rn(__fadd_rn(re, __fmul_rn(b, y0)), __fmul_rn(c, y0))));
    small = __fadd_rn(small, __fadd_rn(ge, __fmul_rn(__fmul_rn(a, d1), d1)));
    float S, Se, t;
    two_sum_rn(one_t1, -t1e, S, Se);
    two_sum_rn(S, -q1, S, t);
    Se = __fadd_rn(Se, t);
    two_sum_rn(S, -q2, S, t);
    Se = __fadd_rn(Se, t);
    two_sum_rn(S, -g, S, t);
    Se = __fadd_rn(Se, t);
    const float e2 = __fadd_rn(S, __fsub_rn(Se, small));
    const float d2 = __fmul_rn(hy0, e2);
    // y0 + d1 + d2 in 62-bit fixed point, rounded once to 53 bits (ties to even)
    const long long Y = fix62(y0) + fix62(d1) + fix62(d2);
    const int lead = 63 - __clzll(Y);                      // 61 or 62
    const int sh = lead - 52;
    unsigned long long man = (unsigned long long)Y >> sh;
    const unsigned long long rem = (unsigned long long)Y & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    int lead2 = lead;
    if (rem > half || (rem == half && (man & 1ull))) {
        man += 1ull;
        if (man >> 53) { man >>= 1; ++lead2; }
    }
    return dbits(((unsigned long long)(lead2 - 62 - k + 1023) << 52) | (man & 0xfffffffffffffull));
}

// 1/x of a double by the same means: Newton-Raphson for the reciprocal (y <- y + y (1 - x y))
// from the single-precision seed, x = m 2^E with m in [1, 2) split into a + b + c, the
// residuals formed exactly as above, y0 + d1 + d2 rounded once to the nearest double; within
// one unit in the last place.  Results outside the normal range (|x| >= 2^1022, a subnormal
// reciprocal), zero, infinities and NaN take the IEEE division.
__device__ __forceinline__ double trcp(double x) {
    const unsigned long long u = ubits(x);
    const int e = (int)(u >> 52) & 0x7ff;
    const unsigned long long mant = u & 0xfffffffffffffull;
    if (e >= 0x7fd || (e == 0 && mant == 0ull)) return 1.0 / x;
    unsigned long long M;
    int E;
    if (e == 0) {
        const int lz = __clzll((long long)mant) - 11;
        M = mant << lz;
        E = -1022 - lz;
    } else {
        M = mant | (1ull << 52);
        E = e - 1023;
    }
    const unsigned A = (unsigned)(M >> 29), B = (unsigned)(M >> 5) & 0xffffffu, Cc = (unsigned)M & 31u;
    const float a = __uint_as_float((127u << 23) | (A & 0x7fffffu));                    // in [1, 2)
    const float b = __fmul_rn(__uint2float_rn(B), 0x1p-47f);
    const float c = __fmul_rn(__uint2float_rn(Cc), 0x1p-52f);
    const float y0 = __fdividef(1.0f, a);
    float t, te;
    two_prod_rn(a, y0, t, te);
    const float one_t = __fsub_rn(1.0f, t);                // exact
    const float e1 = __fsub_rn(one_t, __fadd_rn(te, __fadd_rn(__fmul_rn(b, y0), __fmul_rn(c, y0))));
    const float d1 = __fmul_rn(y0, e1);
    float q1, q1e, q2, q2e;
    two_prod_rn(a, d1, q1, q1e);
    two_prod_rn(b, y0, q2, q2e);
    const float small = __fadd_rn(__fadd_rn(__fadd_rn(q1e, q2e), __fmul_rn(b, d1)),
                                  __fadd_rn(__fmul_rn(c, y0), __fmul_rn(c, d1)));
    float S, Se, tt;
    two_sum_rn(one_t, -te, S, Se);
    two_sum_rn(S, -q1, S, tt);
    Se = __fadd_rn(Se, tt);
    two_sum_rn(S, -q2, S, tt);
    Se = __fadd_rn(Se, tt);
    const float e2 = __fadd_rn(S, __fsub_rn(Se, small));
    const float d2 = __fmul_rn(y0, e2);
    const long long Y = fix62(y0) + fix62(d1) + fix62(d2);
    const int lead = 63 - __clzll(Y);
    const int sh = lead - 52;
    unsigned long long man = (unsigned long long)Y >> sh;
    const unsigned long long rem = (unsigned long long)Y & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    int lead2 = lead;
    if (rem > half || (rem == half && (man & 1ull))) {
        man += 1ull;
        if (man >> 53) { man >>= 1; ++lead2; }
    }
    const int be = lead2 - 62 - E + 1023;
    if (be >= 0x7ff) return 1.0 / x;                       // overflow: the division gives inf
    return dbits((u & ~kMagBits) | ((unsigned long long)be << 52) | (man & 0xfffffffffffffull));
}

// ---------------------------------------------------------------------------------
// Kurganov-Noelle-Petrova update of one node (Sec. 3.2.3 Steps 1-4; readings G1-G7).
// f(i, j): value at node offset (i along x1, j along x2), i, j in [-2, 2].
// ---------------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T minmod3(T a, T b, T c) {
    if (a > T(0) && b > T(0) && c > T(0)) return tmin(a, tmin(b, c));
    if (a < T(0) && b < T(0) && c < T(0)) return tmax(a, tmax(b, c));
    return T(0);
}
// x > 0 for the tests that guard a reciprocal or reciprocal square root of x.  FP32 and
// double words (whose exponent range is FP32's) count x <= 1e-36 as zero, so that 1/x and
// (1/sqrt(x))^2 stay finite; every term this drops is a product with a gradient or a speed
// span of that size, far below the types' rounding.  FP64 tests x > 0 exactly.
template <typename T> __device__ __forceinline__ bool tguard(T x) { return x > T(1e-36f); }
__device__ __forceinline__ bool tguard(double x) { return tpos(x); }
// sqrt(x) for x >= 0
template <typename T> __device__ __forceinline__ T tsqrt(T x) { return tguard(x) ? x * trsqrt(x) : T(0); }

// the same function on bit patterns: when a, b, c are nonzero, not NaN and of one sign, the
// one of least magnitude; else 0
__device__ __forceinline__ double minmod3(double a, double b, double c) {
    const unsigned long long ua = ubits(a), ub = ubits(b), uc = ubits(c);
    const unsigned long long ma = ua & kMagBits, mb = ub & kMagBits, mc = uc & kMagBits;
    const bool ok = ((((ua ^ ub) | (ua ^ uc)) >> 63) == 0) && mag_ok(ma) && mag_ok(mb) && mag_ok(mc);
    double r = (mb < ma) ? b : a;
    const unsigned long long mr = (mb < ma) ? mb : ma;
    r = (mc < mr) ? c : r;
    return ok ? r : 0.0;
}

// |a| < |b| (on bit patterns for FP64)
__device__ __forceinline__ bool tmag_less(float a, float b) { return fabsf(a) < fabsf(b); }
__device__ __forceinline__ bool tmag_less(df a, df b) { return tabs(a) < tabs(b); }
__device__ __forceinline__ bool tmag_less(double a, double b) { return (ubits(a) & kMagBits) < (ubits(b) & kMagBits); }

// one-sided speeds: ap = max(ap, h), am = min(am, h) for ap >= 0 >= am, NaN ignored
template <typename T> __device__ __forceinline__ void speed_range(T h, T& ap, T& am) {
    ap = tmax(ap, h);
    am = tmin(am, h);
}
__device__ __forceinline__ void speed_range(double h, double& ap, double& am) {
    const unsigned long long u = ubits(h), m = u & kMagBits;
    if (mag_ok(m)) {
        if ((u >> 63) == 0) { if (m > ubits(ap)) ap = h; }
        else if (m > (ubits(am) & kMagBits)) am = h;
    }
}

template <typename T>
struct Side {  // one-dimensional limited quadratic on the cell on one side of the node
    T D;  // first difference toward that side, signed as phi_{j+1}-phi_j or phi_j-phi_{j-1}
    T S;  // limited second difference on that cell
};

// x times the limiter parameter theta.  A float product is cheapest; on the FP64 pipe and in
// double words theta = 1 is skipped, and double words apply theta = 2 as an exact scaling.
__device__ __forceinline__ float theta_mul(float x, float theta, int) { return theta * x; }
__device__ __forceinline__ double theta_mul(double x, double theta, int theta_code) {
    if (theta_code == 1) return x;
    if (theta_code == 2) return ttwice(x);
    return theta * x;
}
__device__ __forceinline__ df theta_mul(df x, df theta, int theta_code) {
    if (theta_code == 1) return x;
    if (theta_code == 2) return scale2(x, 2.0f);
    return theta * x;
}

// The update in cell units: with h the cell size, gradients are carried as h * grad (the
// first differences themselves), displacements as d / h, and the time step as dt / h.  The
// one-sided speeds depend only on the gradient's direction, so they are unchanged; every
// formula of Steps 1-4 then holds with h = 1 and dt replaced by dt / h.
template <typename T, typename F>
__device__ __forceinline__ T knp_node(F f, T v0, T dt_h, T theta, int theta_code, int time_level) {
    const T f0 = f(0, 0);
    // Step 1: first differences and limited second differences along x1 and x2
    T dxm3 = f(-1, 0) - f(-2, 0), dxm1 = f0 - f(-1, 0), dxp1 = f(1, 0) - f0, dxp3 = f(2, 0) - f(1, 0);
    T dym3 = f(0, -1) - f(0, -2), dym1 = f0 - f(0, -1), dyp1 = f(0, 1) - f0, dyp3 = f(0, 2) - f(0, 1);
    Side<T> xs[2], ys[2];  // [0] = + side, [1] = - side
    {
        const T c = theta_mul(dxp1 - dxm1, theta, theta_code);  // shared by both limiters
        xs[0].D = dxp1; xs[0].S = minmod3(theta_mul(dxp3 - dxp1, theta, theta_code), thalf(dxp3 - dxm1), c);
        xs[1].D = dxm1; xs[1].S = minmod3(c, thalf(dxp1 - dxm3), theta_mul(dxm1 - dxm3, theta, theta_code));
    }
    {
        const T c = theta_mul(dyp1 - dym1, theta, theta_code);
        ys[0].D = dyp1; ys[0].S = minmod3(theta_mul(dyp3 - dyp1, theta, theta_code), thalf(dyp3 - dym1), c);
        ys[1].D = dym1; ys[1].S = minmod3(c, thalf(dyp1 - dym3), theta_mul(dym1 - dym3, theta, theta_code));
    }
    // one-sided derivatives at the node (times h)
    T px[2] = {xs[0].D - thalf(xs[0].S), xs[1].D + thalf(xs[1].S)};
    T qy[2] = {ys[0].D - thalf(ys[0].S), ys[1].D + thalf(ys[1].S)};
    // Step 2: one-sided speeds over the four pairs (G4; dH/dp = v0 p / |(p,q)|, 0 at the
    // origin).  For a fixed p the magnitude |p| / |(p,q)| falls as |q| grows and keeps its
    // sign, so max(0, .) and min(0, .) of dH/dp over the pairs are attained with the q of
    // least magnitude, and those of dH/dq with the p of least magnitude: the pairs
    // (p0, qm), (p1, qm), (pm, qm'), where qm' is the other q, cover all four.
    const bool tq = tmag_less(qy[1], qy[0]), tp = tmag_less(px[1], px[0]);
    const T qm = tq ? qy[1] : qy[0], qo = tq ? qy[0] : qy[1];
    const T pm = tp ? px[1] : px[0];
    auto inv_norm = [&](T p, T q) -> T {   // v0 / |(p, q)|, 0 at the origin
        const T r2 = p * p + q * q;
        return tguard(r2) ? v0 * trsqrt(r2) : T(0);
    };
    const T r0 = inv_norm(px[0], qm), r1 = inv_norm(px[1], qm), rc = inv_norm(pm, qo);
    T ap = T(0), am = T(0), bp = T(0), bm = T(0);
    speed_range(r0 * px[0], ap, am);
    speed_range(r1 * px[1], ap, am);
    speed_range((tp ? r1 : r0) * qm, bp, bm);   // the pair (pm, qm) is (p0, qm) or (p1, qm)
    speed_range(rc * qo, bp, bm);
    // Step 4 weights (G1, G5): w(s,t) = nx[s] ny[t] / (dxw dyw), one reciprocal
    // FP64: w(s,t) = nx[s] ny[t] / (dxw dyw) with one reciprocal.  FP32 and double words
    // normalise each direction on its own (wx = nx / dxw in [0, 1]), because the product of
    // two small spans leaves their exponent range.
    T nx[2], ny[2], dxw = ap - am, dyw = bp - bm;
    if (tguard(dxw)) { nx[0] = -am; nx[1] = ap; }
    else { nx[0] = T(0.5); nx[1] = T(0.5); dxw = T(1); }
    if (tguard(dyw)) { ny[0] = -bm; ny[1] = bp; }
    else { ny[0] = T(0.5); ny[1] = T(0.5); dyw = T(1); }
    T inv_w = T(1);
    if constexpr (std::is_same<T, double>::value) {
        inv_w = trcp(dxw * dyw);
    } else {
        const T ix = trcp(dxw), iy = trcp(dyw);
        nx[0] = nx[0] * ix; nx[1] = nx[1] * ix;
        ny[0] = ny[0] * iy; ny[1] = ny[1] * iy;
    }
    const T vdt = v0 * dt_h;                 // v0 dt / h
    const T hvdt = thalf(vdt);               // v0 dt / (2 h)
    // Step 3: values at the four intermediate points (G2, G3).  Along each direction the
    // limited quadratic on the side's cell, in cell units: with e the displacement / h and
    // sg = -1 on the + side, +1 on the - side,  X(e) = D e + S e (e + sg) / 2 and
    // h X'(e) = D + S (e + sg / 2).
    T Y[2], dY[2], ey[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        ey[t] = (t == 0 ? bp : bm) * dt_h;
        const T sgn = (t == 0) ? T(-1) : T(1);
        Y[t] = ey[t] * (ys[t].D + thalf(ys[t].S) * (ey[t] + sgn));
        dY[t] = ys[t].D + ys[t].S * (ey[t] + thalf(sgn));
    }
    T acc = T(0);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int cx = (s == 0) ? 1 : -1;
        const T ex = (s == 0 ? ap : am) * dt_h;
        const T Dx = xs[s].D, Sx = xs[s].S;
        const T sgn = (s == 0) ? T(-1) : T(1);
        const T X = ex * (Dx + thalf(Sx) * (ex + sgn));
        const T dX = Dx + Sx * (ex + thalf(sgn));
        const T fx0 = (s == 0) ? Dx : -Dx;   // f(cx, 0) - f0, the side's first difference
        T accs = T(0);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int cy = (t == 0) ? 1 : -1;
            // mixed second difference of the quadrant cell (h^2 times the bilinear cross term)
            const T mixed = (f(cx, cy) - f(0, cy)) - fx0;
            const T cross = (cx * cy > 0) ? mixed : -mixed;
            const T val = X + Y[t] + cross * ex * ey[t];   // minus f0, added once below
            T p = dX + cross * ey[t];
            T q = dY[t] + cross * ex;
            if (time_level == 0) {
                // (p, q) -= dt/2 Hess grad_(p,q) H, grad H = v0 (p, q) / |(p, q)|
                const T r2 = p * p + q * q;
                if (tguard(r2)) {
                    const T w = hvdt * trsqrt(r2);
                    const T np = p - w * (Sx * p + cross * q);
                    const T nq = q - w * (cross * p + ys[t].S * q);
                    p = np; q = nq;
                }
            }
            const T s2 = p * p + q * q;
            const T g = tguard(s2) ? s2 * trsqrt(s2) : T(0);   // h |grad|
            const T psi = val - vdt * g;
            accs += ny[t] * psi;
        }
        acc += nx[s] * accs;
    }
    return f0 + acc * inv_w;   // the weights sum to one
}

// ---------------------------------------------------------------------------------
// Packed FP32 pairs.  Blackwell issues two FP32 additions, multiplications or fused
// multiply-adds as one instruction (add/sub/mul/fma .rn.f32x2), each lane rounded exactly
// as the scalar operation.  The FP32 stencil updates two nodes at once in the two lanes:
// every lane's result is the one the same operations give on that node alone, so it does
// not depend on which node shares its pair.  Comparisons, min/max, selects and the
// special-function reciprocal (square root) stay per lane.
// ---------------------------------------------------------------------------------
struct f2 { float x, y; };
__device__ __forceinline__ f2 mkf2(float a, float b) { f2 r; r.x = a; r.y = b; return r; }
__device__ __forceinline__ f2 bcast(float a) { return mkf2(a, a); }
__device__ __forceinline__ unsigned long long pk2(f2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ f2 upk2(unsigned long long v) {
    f2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ f2 operator+(f2 a, f2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)));
    return upk2(r);
}
__device__ __forceinline__ f2 operator-(f2 a, f2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)));
    return upk2(r);
}
__device__ __forceinline__ f2 operator*(f2 a, f2 b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)));
    return upk2(r);
}
__device__ __forceinline__ f2 operator-(f2 a) { return mkf2(-a.x, -a.y); }
// a b + c, one rounding per lane
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)), "l"(pk2(c)));
    return upk2(r);
}
__device__ __forceinline__ f2 sel2(bool cx, bool cy, f2 a, f2 b) { return mkf2(cx ? a.x : b.x, cy ? a.y : b.y); }
__device__ __forceinline__ f2 fmax2(f2 a, f2 b) { return mkf2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
__device__ __forceinline__ f2 fmin2(f2 a, f2 b) { return mkf2(fminf(a.x, b.x), fminf(a.y, b.y)); }

// minmod of three floats: the argument of least magnitude when all three are nonzero and of
// one sign, else zero; computed from the magnitudes' minimum and the sign bits
__device__ __forceinline__ float minmod3_bits(float a, float b, float c) {
    const unsigned ua = __float_as_uint(a), ub = __float_as_uint(b), uc = __float_as_uint(c);
    const float m = fminf(fminf(fabsf(a), fabsf(b)), fabsf(c));
    const bool agree = (((ua ^ ub) | (ua ^ uc)) & 0x80000000u) == 0u;
    return agree ? __uint_as_float(__float_as_uint(m) | (ua & 0x80000000u)) : 0.0f;
}
__device__ __forceinline__ f2 minmod3(f2 a, f2 b, f2 c) {
    return mkf2(minmod3_bits(a.x, b.x, c.x), minmod3_bits(a.y, b.y, c.y));
}
// v / |(p, q)| per lane from r2 = p^2 + q^2, zero at the origin (guarded as tguard)
__device__ __forceinline__ f2 scaled_rsqrt2(f2 r2, f2 v) {
    return mkf2(tguard(r2.x) ? v.x * rsqrtf(r2.x) : 0.0f, tguard(r2.y) ? v.y * rsqrtf(r2.y) : 0.0f);
}

// The KNP update of two nodes (Sec. 3.2.3 Steps 1-4, readings G1-G7), in cell units as
// knp_node, for FP32 fields given as differences to each node's own value: f(i, j) returns
// the pair (U(node a + (i, j)) - U(a), U(node b + (i, j)) - U(b)), so f(0, 0) = 0; returns
// the two increments U^{n+1} - U^n.
template <typename F>
__device__ __forceinline__ f2 knp_node_x2(F f, f2 v0, float dt_h, float theta, int time_level) {
    const f2 th = bcast(theta), hf = bcast(0.5f);
    // Step 1: first differences (f(0, 0) = 0) and limited second differences
    const f2 xm1 = f(-1, 0), xp1 = f(1, 0), ym1 = f(0, -1), yp1 = f(0, 1);
    const f2 dxm3 = xm1 - f(-2, 0), dxm1 = -xm1, dxp1 = xp1, dxp3 = f(2, 0) - xp1;
    const f2 dym3 = ym1 - f(0, -2), dym1 = -ym1, dyp1 = yp1, dyp3 = f(0, 2) - yp1;
    const f2 cxl = th * (dxp1 - dxm1), cyl = th * (dyp1 - dym1);
    const f2 Sxp = minmod3(th * (dxp3 - dxp1), hf * (dxp3 - dxm1), cxl);
    const f2 Sxm = minmod3(cxl, hf * (dxp1 - dxm3), th * (dxm1 - dxm3));
    const f2 Syp = minmod3(th * (dyp3 - dyp1), hf * (dyp3 - dym1), cyl);
    const f2 Sym = minmod3(cyl, hf * (dyp1 - dym3), th * (dym1 - dym3));
    // one-sided derivatives at the node (times h)
    const f2 px0 = fma2(-hf, Sxp, dxp1), px1 = fma2(hf, Sxm, dxm1);
    const f2 qy0 = fma2(-hf, Syp, dyp1), qy1 = fma2(hf, Sym, dym1);
    // Step 2: one-sided speeds over the four pairs, from the three pairs that attain the
    // extremes (the q of least magnitude for dH/dp, the p of least magnitude for dH/dq)
    const bool tqx = fabsf(qy1.x) < fabsf(qy0.x), tqy = fabsf(qy1.y) < fabsf(qy0.y);
    const bool tpx = fabsf(px1.x) < fabsf(px0.x), tpy = fabsf(px1.y) < fabsf(px0.y);
    const f2 qm = sel2(tqx, tqy, qy1, qy0), qo = sel2(tqx, tqy, qy0, qy1), pm = sel2(tpx, tpy, px1, px0);
    const f2 r0 = scaled_rsqrt2(fma2(px0, px0, qm * qm), v0);
    const f2 r1 = scaled_rsqrt2(fma2(px1, px1, qm * qm), v0);
    const f2 rc = scaled_rsqrt2(fma2(pm, pm, qo * qo), v0);
    const f2 z = bcast(0.0f);
    const f2 hp0 = r0 * px0, hp1 = r1 * px1, hq0 = sel2(tpx, tpy, r1, r0) * qm, hq1 = rc * qo;
    const f2 ap = fmax2(fmax2(z, hp0), hp1), am = fmin2(fmin2(z, hp0), hp1);
    const f2 bp = fmax2(fmax2(z, hq0), hq1), bm = fmin2(fmin2(z, hq0), hq1);
    // Step 4 weights (G1, G5), each direction normalised on its own
    f2 dxw = ap - am, dyw = bp - bm;
    const bool gx0 = tguard(dxw.x), gx1 = tguard(dxw.y), gy0 = tguard(dyw.x), gy1 = tguard(dyw.y);
    const f2 ix = mkf2(gx0 ? trcp(dxw.x) : 1.0f, gx1 ? trcp(dxw.y) : 1.0f);
    const f2 iy = mkf2(gy0 ? trcp(dyw.x) : 1.0f, gy1 ? trcp(dyw.y) : 1.0f);
    const f2 nx[2] = {sel2(gx0, gx1, -am, hf) * ix, sel2(gx0, gx1, ap, hf) * ix};
    const f2 ny[2] = {sel2(gy0, gy1, -bm, hf) * iy, sel2(gy0, gy1, bp, hf) * iy};
    const f2 dth = bcast(dt_h);
    const f2 vdt = v0 * dth;          // v0 dt / h
    const f2 hvdt = hf * vdt;         // v0 dt / (2 h)
    // Step 3: values at the four intermediate points (G2, G3), the limited quadratics of
    // each side in cell units: X(e) = D e + S e (e + sg) / 2, h X'(e) = D + S (e + sg / 2)
    const f2 Dy[2] = {dyp1, dym1}, Sy[2] = {Syp, Sym};
    f2 Y[2], dY[2], ey[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const float sg = (t == 0) ? -1.0f : 1.0f;
        ey[t] = (t == 0 ? bp : bm) * dth;
        Y[t] = fma2(Dy[t], ey[t], hf * ((Sy[t] * ey[t]) * (ey[t] + bcast(sg))));
        dY[t] = fma2(Sy[t], ey[t] + bcast(0.5f * sg), Dy[t]);
    }
    const f2 Dx[2] = {dxp1, dxm1}, Sxs[2] = {Sxp, Sxm};
    f2 acc = z;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int cx = (s == 0) ? 1 : -1;
        const float sg = (s == 0) ? -1.0f : 1.0f;
        const f2 ex = (s == 0 ? ap : am) * dth;
        const f2 X = fma2(Dx[s], ex, hf * ((Sxs[s] * ex) * (ex + bcast(sg))));
        const f2 dX = fma2(Sxs[s], ex + bcast(0.5f * sg), Dx[s]);
        const f2 fx = f(cx, 0);
        f2 accs = z;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int cy = (t == 0) ? 1 : -1;
            // h^2 times the bilinear cross term of the quadrant cell
            const f2 mixed = (f(cx, cy) - f(0, cy)) - fx;
            const f2 cross = (cx * cy > 0) ? mixed : -mixed;
            const f2 val = fma2(cross * ex, ey[t], X + Y[t]);
            f2 p = fma2(cross, ey[t], dX);
            f2 q = fma2(cross, ex, dY[t]);
            if (time_level == 0) {
                // (p, q) -= dt/2 Hess grad_(p,q) H, grad H = v0 (p, q) / |(p, q)|
                const f2 w = scaled_rsqrt2(fma2(p, p, q * q), -hvdt);
                const f2 np = fma2(w, fma2(Sxs[s], p, cross * q), p);
                const f2 nq = fma2(w, fma2(cross, p, Sy[t] * q), q);
                p = np;
                q = nq;
            }
            const f2 s2 = fma2(p, p, q * q);
            const f2 g = mkf2(tguard(s2.x) ? s2.x * rsqrtf(s2.x) : 0.0f, tguard(s2.y) ? s2.y * rsqrtf(s2.y) : 0.0f);
            accs = fma2(ny[t], fma2(-vdt, g, val), accs);
        }
        acc = fma2(nx[s], accs, acc);
    }
    return acc;
}

// ---------------------------------------------------------------------------------
// Packed double words: two double-word values, one per lane of the packed FP32 instructions.
// Every operation is the one of fdm_df.cuh (TwoSum, FastTwoSum, FMA TwoProd, the sloppy
// double-word sum and the double-word product of Joldes, Muller & Popescu), carried out on
// both lanes by one instruction, each lane rounded as the scalar operation is, so a lane's
// result equals the scalar double-word result bit for bit.
// ---------------------------------------------------------------------------------
struct df2 { f2 hi, lo; };
__device__ __forceinline__ df lane(const df2& v, int i) { return i == 0 ? df(v.hi.x, v.lo.x) : df(v.hi.y, v.lo.y); }
__device__ __forceinline__ df2 mkdf2(df a, df b) { df2 r; r.hi = mkf2(a.hi, b.hi); r.lo = mkf2(a.lo, b.lo); return r; }
__device__ __forceinline__ df2 bcast2(df a) { return mkdf2(a, a); }
__device__ __forceinline__ void two_sum2(f2 a, f2 b, f2& s, f2& e) {
    s = a + b;
    const f2 bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum2(f2 a, f2 b, f2& s, f2& e) {   // |a| >= |b|
    s = a + b;
    e = b - (s - a);
}
__device__ __forceinline__ df2 operator+(df2 x, df2 y) {
    f2 sh, sl, zh, zl;
    two_sum2(x.hi, y.hi, sh, sl);
    const f2 v = x.lo + y.lo;
    const f2 w = sl + v;
    fast_two_sum2(sh, w, zh, zl);
    df2 r;
    r.hi = zh;
    r.lo = zl;
    return r;
}
__device__ __forceinline__ df2 operator-(df2 x) { df2 r; r.hi = -x.hi; r.lo = -x.lo; return r; }
__device__ __forceinline__ df2 operator-(df2 x, df2 y) { return x + (-y); }
__device__ __forceinline__ df2 operator*(df2 x, df2 y) {
    const f2 ch = x.hi * y.hi;
    const f2 cl1 = fma2(x.hi, y.hi, -ch);
    const f2 tl0 = x.lo * y.lo;
    const f2 tl1 = fma2(x.hi, y.lo, tl0);
    const f2 cl2 = fma2(x.lo, y.hi, tl1);
    const f2 cl3 = cl1 + cl2;
    df2 r;
    fast_two_sum2(ch, cl3, r.hi, r.lo);
    return r;
}
__device__ __forceinline__ df2 mul_f2(df2 x, f2 y) {
    const f2 ch = x.hi * y;
    const f2 cl1 = fma2(x.hi, y, -ch);
    const f2 cl3 = fma2(x.lo, y, cl1);
    df2 r;
    fast_two_sum2(ch, cl3, r.hi, r.lo);
    return r;
}
__device__ __forceinline__ df2 scale2x(df2 x, float p2) { df2 r; r.hi = x.hi * bcast(p2); r.lo = x.lo * bcast(p2); return r; }
__device__ __forceinline__ df2 thalf(df2 x) { return scale2x(x, 0.5f); }
// reciprocal and reciprocal square root: the float seeds per lane, the Newton step packed
__device__ __forceinline__ df2 trcp(df2 y) {
    const f2 r0 = mkf2(rcp_seed(y.hi.x), rcp_seed(y.hi.y));
    const df2 p = mul_f2(y, r0);
    const f2 e = (bcast(1.0f) - p.hi) - p.lo;
    df2 r;
    two_sum2(r0, r0 * e, r.hi, r.lo);
    return r;
}
__device__ __forceinline__ df2 trsqrt(df2 x) {
    const f2 r0 = mkf2(rsqrt_seed(x.hi.x), rsqrt_seed(x.hi.y));
    const f2 q = r0 * r0;
    const f2 qe = fma2(r0, r0, -q);
    df2 qq;
    qq.hi = q;
    qq.lo = qe;
    const df2 h = x * qq;
    const f2 e = (bcast(1.0f) - h.hi) - h.lo;
    df2 r;
    two_sum2(r0, (bcast(0.5f) * r0) * e, r.hi, r.lo);
    return r;
}
__device__ __forceinline__ df2 sel2(bool ca, bool cb, df2 a, df2 b) {
    df2 r;
    r.hi = sel2(ca, cb, a.hi, b.hi);
    r.lo = sel2(ca, cb, a.lo, b.lo);
    return r;
}
__device__ __forceinline__ df2 minmod3(df2 a, df2 b, df2 c) {
    return mkdf2(minmod3(lane(a, 0), lane(b, 0), lane(c, 0)), minmod3(lane(a, 1), lane(b, 1), lane(c, 1)));
}
__device__ __forceinline__ df2 theta_mul(df2 x, df theta, int theta_code) {
    if (theta_code == 1) return x;
    if (theta_code == 2) return scale2x(x, 2.0f);
    return bcast2(theta) * x;
}
__device__ __forceinline__ void speed_range(df2 h, df2& ap, df2& am) {
    df a0 = lane(ap, 0), a1 = lane(ap, 1), m0 = lane(am, 0), m1 = lane(am, 1);
    speed_range(lane(h, 0), a0, m0);
    speed_range(lane(h, 1), a1, m1);
    ap = mkdf2(a0, a1);
    am = mkdf2(m0, m1);
}

// knp_node for two nodes of double-word fields at once (one per lane): the same operations
// in the same order as knp_node<df>, so each lane is that function's result bit for bit;
// per-lane decisions (limiter, speeds, guards) become selects.
template <typename F>
__device__ __forceinline__ df2 knp_node_df2(F f, df2 v0, df dt_h, df theta, int theta_code, int time_level) {
    const df2 f0 = f(0, 0);
    const df2 dxm3 = f(-1, 0) - f(-2, 0), dxm1 = f0 - f(-1, 0), dxp1 = f(1, 0) - f0, dxp3 = f(2, 0) - f(1, 0);
    const df2 dym3 = f(0, -1) - f(0, -2), dym1 = f0 - f(0, -1), dyp1 = f(0, 1) - f0, dyp3 = f(0, 2) - f(0, 1);
    df2 xD[2], xS[2], yD[2], yS[2];   // [0] = + side, [1] = - side
    {
        const df2 c = theta_mul(dxp1 - dxm1, theta, theta_code);
        xD[0] = dxp1; xS[0] = minmod3(theta_mul(dxp3 - dxp1, theta, theta_code), thalf(dxp3 - dxm1), c);
        xD[1] = dxm1; xS[1] = minmod3(c, thalf(dxp1 - dxm3), theta_mul(dxm1 - dxm3, theta, theta_code));
    }
    {
        const df2 c = theta_mul(dyp1 - dym1, theta, theta_code);
        yD[0] = dyp1; yS[0] = minmod3(theta_mul(dyp3 - dyp1, theta, theta_code), thalf(dyp3 - dym1), c);
        yD[1] = dym1; yS[1] = minmod3(c, thalf(dyp1 - dym3), theta_mul(dym1 - dym3, theta, theta_code));
    }
    const df2 px[2] = {xD[0] - thalf(xS[0]), xD[1] + thalf(xS[1])};
    const df2 qy[2] = {yD[0] - thalf(yS[0]), yD[1] + thalf(yS[1])};
    bool tq[2], tp[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        tq[i] = tmag_less(lane(qy[1], i), lane(qy[0], i));
        tp[i] = tmag_less(lane(px[1], i), lane(px[0], i));
    }
    const df2 qm = sel2(tq[0], tq[1], qy[1], qy[0]), qo = sel2(tq[0], tq[1], qy[0], qy[1]);
    const df2 pm = sel2(tp[0], tp[1], px[1], px[0]);
    const df2 zero = bcast2(df(0.0f)), half = bcast2(df(0.5f)), one = bcast2(df(1.0f));
    auto inv_norm = [&](df2 p, df2 q) -> df2 {   // v0 / |(p, q)|, 0 at the origin
        const df2 r2 = p * p + q * q;
        return sel2(tguard(lane(r2, 0)), tguard(lane(r2, 1)), v0 * trsqrt(r2), zero);
    };
    const df2 r0 = inv_norm(px[0], qm), r1 = inv_norm(px[1], qm), rc = inv_norm(pm, qo);
    df2 ap = zero, am = zero, bp = zero, bm = zero;
    speed_range(r0 * px[0], ap, am);
    speed_range(r1 * px[1], ap, am);
    speed_range(sel2(tp[0], tp[1], r1, r0) * qm, bp, bm);
    speed_range(rc * qo, bp, bm);
    df2 dxw = ap - am, dyw = bp - bm;
    const bool gx0 = tguard(lane(dxw, 0)), gx1 = tguard(lane(dxw, 1));
    const bool gy0 = tguard(lane(dyw, 0)), gy1 = tguard(lane(dyw, 1));
    df2 nx[2] = {sel2(gx0, gx1, -am, half), sel2(gx0, gx1, ap, half)};
    df2 ny[2] = {sel2(gy0, gy1, -bm, half), sel2(gy0, gy1, bp, half)};
    dxw = sel2(gx0, gx1, dxw, one);
    dyw = sel2(gy0, gy1, dyw, one);
    const df2 ix = trcp(dxw), iy = trcp(dyw);
    nx[0] = nx[0] * ix; nx[1] = nx[1] * ix;
    ny[0] = ny[0] * iy; ny[1] = ny[1] * iy;
    const df2 dth = bcast2(dt_h);
    const df2 vdt = v0 * dth;
    const df2 hvdt = thalf(vdt);
    df2 Y[2], dY[2], ey[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        ey[t] = (t == 0 ? bp : bm) * dth;
        const df2 sgn = bcast2(df((t == 0) ? -1.0f : 1.0f));
        Y[t] = ey[t] * (yD[t] + thalf(yS[t]) * (ey[t] + sgn));
        dY[t] = yD[t] + yS[t] * (ey[t] + thalf(sgn));
    }
    df2 acc = zero;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int cx = (s == 0) ? 1 : -1;
        const df2 ex = (s == 0 ? ap : am) * dth;
        const df2 Dx = xD[s], Sx = xS[s];
        const df2 sgn = bcast2(df((s == 0) ? -1.0f : 1.0f));
        const df2 X = ex * (Dx + thalf(Sx) * (ex + sgn));
        const df2 dX = Dx + Sx * (ex + thalf(sgn));
        const df2 fx0 = (s == 0) ? Dx : -Dx;   // f(cx, 0) - f0, the side's first difference
        df2 accs = zero;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int cy = (t == 0) ? 1 : -1;
            const df2 mixed = (f(cx, cy) - f(0, cy)) - fx0;
            const df2 cross = (cx * cy > 0) ? mixed : -mixed;
            const df2 val = X + Y[t] + cross * ex * ey[t];   // minus f0, added once below
            df2 p = dX + cross * ey[t];
            df2 q = dY[t] + cross * ex;
            if (time_level == 0) {
                const df2 r2 = p * p + q * q;
                const bool g0 = tguard(lane(r2, 0)), g1 = tguard(lane(r2, 1));
                const df2 w = hvdt * trsqrt(r2);
                const df2 np = p - w * (Sx * p + cross * q);
                const df2 nq = q - w * (cross * p + yS[t] * q);
                p = sel2(g0, g1, np, p);
                q = sel2(g0, g1, nq, q);
            }
            const df2 s2 = p * p + q * q;
            const df2 g = sel2(tguard(lane(s2, 0)), tguard(lane(s2, 1)), s2 * trsqrt(s2), zero);
            const df2 psi = val - vdt * g;
            accs = accs + ny[t] * psi;
        }
        acc = acc + nx[s] * accs;
    }
    return f0 + acc;   // the weights sum to one
}

}  // namespace fdm
