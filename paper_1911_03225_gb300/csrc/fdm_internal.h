// fdm_internal.h -- structures shared by the C-ABI layer and the kernels.
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

#include "../../include/fdm.h"

namespace fdm {

// Per-handle scalars in device memory; every per-step quantity lives here so that a step
// is a fixed launch sequence (capturable in a CUDA graph).
struct fdm_dev_scalars {
    unsigned long long vmax_bits;  // max |v0| of the current step, bits of a double >= 0
    unsigned int done_count;       // blocks of the stencil kernel that have finished
    int status;                    // fdm_status of device-side checks
    long long step;                // steps since the last fdm_set_*
    double t, dt, max_abs_v0;
    double mean_up13, eps_bar13, sigma_bar13;  // state at the start of the current step
    double phi_ref;                // mixed precision: U13 = phi_ref + stored value
    int cur;                       // state buffer holding U13 (0 or 1); flipped by each step
    unsigned int ri_count;         // blocks of the inverse row kernel that have finished
    long long steps_left;          // gated (batched) launches: steps this instance may still take
    double dt_next, dt_h_next;     // dt of the step being taken and dt / dx (set with max |v0|)
};

constexpr int kKernelsPerStep = 4;
constexpr int kKnpShapes = 4;  // stencil block shapes per precision (shape 0 = default)

struct LaunchGeom {
    int R;             // rows per block of the row kernels
    int C;             // spectral columns per block of the column kernel
    size_t row_smem, col_smem;
    int row_blocks, col_blocks;
    int row_threads, col_threads;  // threads per block of the row / column FFT kernels
    int knp_shape;     // stencil block shape, index in [0, kKnpShapes)
    int tuned;         // chosen by the autotuner
    double kernel_us[kKernelsPerStep];  // tuned: best time of each step kernel
};

// One group of `count` instances with identical parameters.  Every buffer holds `count`
// consecutive instances (instance i at offset i * n, spectra at i * n/2 complex).
struct Dev {
    fdm_params p;          // validated copy (nz resolved)
    LaunchGeom geom;
    int count;             // instances in the group
    int gated;             // step launches honour each instance's steps_left (batches)
    void* phi[2];          // double-buffered U13 (type T); the current one is sc[i].cur
    void* phi_lo[2];       // FDM_MIXED: low FP32 words of U13 (U13 = phi + phi_lo); else null
    void* mfac;            // T [count][n]: mobility factor m(x) of the celerity, or null (m = 1)
    void* tau;             // T
    void* spec;            // cpx<T> [n1/2][n2] per instance
    void* spec2;           // cpx<T> [n1/2][n2] (single instance only; readouts)
    void* Kh;              // T [n1/2+1][n2/2+1]
    void* tw1;             // cpx<T> [n1]: exp(-2 pi i m / n1), for the real/half-complex twists
    void* tw2;             // cpx<T> [n2]
    void* pt1;             // cpx<T> pass twiddle tables of the n1/2-point row transform
    void* pt2;             // cpx<T> pass twiddle tables of the n2-point column transform
    double* row_partials;  // [count][n2]: FP64 sum of each row of U13
    double* red;           // reduction partials [6 * red_blocks]
    double* red_host;      // pinned host copy: the instance's scalars, then the partials
    int red_blocks;
    fdm_dev_scalars* sc;   // [count]
    double phi_ref_host;   // single instance: host copy of sc[0].phi_ref
};

// Launch shapes: R rows per row-kernel block and C columns per column-kernel block (0:
// heuristic choice), stencil shape index.  Candidate lists hold every valid R or C.
template <typename T> LaunchGeom geometry(int n1, int n2, int R = 0, int C = 0, int knp_shape = 0);
template <typename T> int row_candidates(int n1, int n2, int* out, int max);
template <typename T> int col_candidates(int n1, int n2, int* out, int max);
template <typename T> void knp_shape_info(int shape, int* ty, int* npt, int* minb);
// Times the candidate shapes on the group's buffers (their contents are overwritten) and
// stores the fastest in d.geom; results are cached per device, precision, grid, instance
// count and scheme variant.  Leaves the scalars of every instance zeroed.
template <typename T> cudaError_t autotune_group(Dev& d, cudaStream_t s);
// fill U13 (buffer 0 of every instance) with a smooth synthetic field with kinks
template <typename T> void launch_tune_fill(const Dev& d, cudaStream_t s);
template <typename T> cudaError_t configure_kernels();
// step launches read U13 from phi[sc[i].cur] of every instance and write the other buffer
template <typename T> void launch_step(const Dev& d, cudaStream_t s);
template <typename T> void launch_phase(const Dev& d, int phase, cudaStream_t s);
template <typename T> void launch_static(const Dev& d, cudaStream_t s);
template <typename T> void launch_static_to(const Dev& d, T* dst, cudaStream_t s);
// stress component comp (Voigt order 11, 22, 33, 23, 13, 12; not 13, which takes
// launch_static_to with its macroscopic stress) with the plane table in d.Kh
template <typename T> void launch_stress_to(const Dev& d, int comp, T* dst, cudaStream_t s);
// unnormalised 2-D transforms of one real field (packed transposed spectrum of n/2 complex)
template <typename T> void launch_fft_forward(const Dev& d, const T* src, void* spec, cudaStream_t s);
template <typename T> void launch_fft_inverse(const Dev& d, void* spec, T* dst, cudaStream_t s);
// the same for `count` consecutive fields of the group's grid (spectra consecutive too)
template <typename T> void launch_fft_forward_many(const Dev& d, const T* src, void* spec, int count, cudaStream_t s);
template <typename T> void launch_fft_inverse_many(const Dev& d, void* spec, T* dst, int count, cudaStream_t s);
// the step's time step (single instance) from a tau13 already in d.tau: max |v0| and dt
template <typename T> void launch_celerity_dt(const Dev& d, cudaStream_t s);
template <typename T> void launch_alpha(const Dev& d, const T* phi, T* a11, T* a12, cudaStream_t s);
template <typename T>
void launch_curl_inverse(const Dev& d, const T* a11, const T* a12, T* phi_out, double mean_up13, double phi_ref,
                         double* partials, int nblk, cudaStream_t s);
template <typename T> void launch_convert(const double* a, T* b, size_t n, double offset, cudaStream_t s);
// sums of the Nye components of the current state of instance inst (buffer sc[inst].cur)
template <typename T> void launch_alpha_sums(const Dev& d, int inst, double* partials, int nblk, cudaStream_t s);
template <typename T>
void launch_velocity(const Dev& d, const T* a11, const T* a12, const T* tau, const T* phi, T* v1, T* v2,
                     cudaStream_t s);
void launch_pair_to_double(const float* hi, const float* lo, double* out, size_t n, cudaStream_t s);
// U13 of the current state (FP64) against prev[n]: partials[2 nblk] = per block sum of
// (U - prev)^2 and of prev^2, then prev <- U; first = 1 only copies
template <typename T>
void launch_state_change(const Dev& d, double* prev, int first, double* partials, int nblk, cudaStream_t s);
// twiddles exp(-2 pi i m / n) into tw (cpx<T> [n]) and the pass tables of an L-point
// transform into pt (cpx<T> [pass_table_len(L)]); either may be null
template <typename T> void launch_twiddle_tables(void* tw, int n, void* pt, int L, cudaStream_t s);
// |chi-hat(k3)|^2 of a layer of nh voxels in a cell of nz, k3 in [0, nz/2] (double [nz/2 + 1])
void launch_layer_weights(double* w3, int nz, int nh, cudaStream_t s);
void launch_kernel_table(double* Kh, int n1, int n2, int nz, int nh, double mu, double nu, const double* w3,
                         cudaStream_t s);
void launch_stress_table(double* Kh, int n1, int n2, int nz, int comp, double mu, double nu, const double* w3,
                         cudaStream_t s);

// Persistent batched step (mixed precision groups): every phase of every group in one
// cooperative launch of resident blocks, phases separated by a bounded grid barrier.
constexpr int kPersistThreads = 512;
struct PersistBarrier {
    unsigned int count;       // arrivals in the current round
    unsigned int gen;         // completed rounds
    int status;               // FDM_OK, or FDM_ERR_TIMEOUT once a wait gave up
    int extra;                // arrivals expected beyond the grid (a test hook; 0 normally)
    long long limit_cycles;   // a barrier wait gives up after this many SM clock cycles
};
// bytes of one group descriptor; fills host_desc[ngroups] (FDM_ERR_INVALID_ARG unless every
// group is FDM_MIXED with n1 >= 32) and the dynamic shared memory the launch needs
size_t persist_group_bytes();
fdm_status persist_prepare(const Dev* const* groups, int ngroups, void* host_desc, size_t* smem);
// dev_desc: the descriptors in device memory; bar: reset by the caller (count, status = 0)
cudaError_t persist_launch(const void* dev_desc, int ngroups, int nsteps, PersistBarrier* bar, size_t smem,
                           cudaStream_t s);

struct df;  // double-word type (fdm_df.cuh)

// Runs BODY with T bound to the storage/arithmetic type of precision PREC.
#define FDM_DISPATCH(PREC, BODY)                                      \
    do {                                                              \
        if ((PREC) == FDM_MIXED) { using T = float; BODY; }           \
        else if ((PREC) == FDM_DF64) { using T = ::fdm::df; BODY; }   \
        else { using T = double; BODY; }                              \
    } while (0)

}  // namespace fdm
