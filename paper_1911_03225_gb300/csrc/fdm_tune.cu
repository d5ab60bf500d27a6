// fdm_tune.cu -- launch-shape autotuner of the step kernels.
//
// Each of the four kernels of a step admits several launch shapes: rows per block of the
// two row FFT kernels, spectral columns per block of the column kernel, and the block shape
// of the stencil.  All shapes compute bit-identical values (the per-row, per-column and
// per-node arithmetic and every reduction order are independent of them), so the choice is
// purely one of speed, and the fastest depends on the grid, the precision, the instances
// per launch and the GPU.  At creation a group therefore times every candidate on its own
// buffers, filled with a synthetic field, and keeps the fastest shape for each kernel.
// Choices are cached for the process per (device, precision, grid, instances, scheme
// variant), so later groups of the same kind start without timing.  If the environment
// variable FDM_TUNE_CACHE names a file, choices also persist across processes there, one
// JSON object per line keyed by the GPU's name and SM count; lines that do not parse or
// name shapes this library does not offer are ignored.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "fdm_df.cuh"
#include "fdm_internal.h"

namespace fdm {
namespace {

using TuneKey = std::tuple<int, int, int, int, int, int, int, int, int>;
std::mutex g_tune_mutex;
std::map<TuneKey, LaunchGeom> g_tune_cache;

template <typename T> constexpr int prec_code();
template <> constexpr int prec_code<double>() { return FDM_FP64; }
template <> constexpr int prec_code<float>() { return FDM_MIXED; }
template <> constexpr int prec_code<df>() { return FDM_DF64; }

// ---- persistent cache (FDM_TUNE_CACHE)
struct FileKey {
    std::string gpu;
    int sms, prec, n1, n2, count, gated, tl, vm, fr;
    bool operator<(const FileKey& o) const {
        return std::tie(gpu, sms, prec, n1, n2, count, gated, tl, vm, fr) <
               std::tie(o.gpu, o.sms, o.prec, o.n1, o.n2, o.count, o.gated, o.tl, o.vm, o.fr);
    }
};
struct FileVal {
    int R, C, shape;
    double us[kKernelsPerStep];
};
bool g_file_loaded = false;
std::map<FileKey, FileVal> g_file_cache;

const char* cache_path() {
    const char* p = std::getenv("FDM_TUNE_CACHE");
    return (p && *p) ? p : nullptr;
}

bool device_identity(int dev, std::string* name, int* sms) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    name->assign(prop.name);
    for (char& c : *name)
        if (c == '"' || c == '\\') c = '_';
    *sms = prop.multiProcessorCount;
    return true;
}

// reads the cache file once (caller holds g_tune_mutex)
void load_file_cache() {
    if (g_file_loaded) return;
    g_file_loaded = true;
    const char* path = cache_path();
    if (!path) return;
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    char line[1024], gpu[256];
    while (std::fgets(line, sizeof line, f)) {
        FileKey k;
        FileVal v;
        int n = std::sscanf(line,
                            "{\"gpu\": \"%255[^\"]\", \"sms\": %d, \"precision\": %d, \"n1\": %d, \"n2\": %d, "
                            "\"instances\": %d, \"gated\": %d, \"time_level\": %d, \"velocity_mode\": %d, "
                            "\"friction\": %d, \"rows\": %d, \"cols\": %d, \"stencil_shape\": %d, "
                            "\"kernel_us\": [%lf, %lf, %lf, %lf]}",
                            gpu, &k.sms, &k.prec, &k.n1, &k.n2, &k.count, &k.gated, &k.tl, &k.vm, &k.fr, &v.R, &v.C,
                            &v.shape, &v.us[0], &v.us[1], &v.us[2], &v.us[3]);
        if (n != 17) continue;
        k.gpu = gpu;
        g_file_cache[k] = v;
    }
    std::fclose(f);
}

void append_file_cache(const FileKey& k, const FileVal& v) {
    const char* path = cache_path();
    if (!path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f,
                 "{\"gpu\": \"%s\", \"sms\": %d, \"precision\": %d, \"n1\": %d, \"n2\": %d, \"instances\": %d, "
                 "\"gated\": %d, \"time_level\": %d, \"velocity_mode\": %d, \"friction\": %d, \"rows\": %d, "
                 "\"cols\": %d, \"stencil_shape\": %d, \"kernel_us\": [%.3f, %.3f, %.3f, %.3f]}\n",
                 k.gpu.c_str(), k.sms, k.prec, k.n1, k.n2, k.count, k.gated, k.tl, k.vm, k.fr, v.R, v.C, v.shape,
                 v.us[0], v.us[1], v.us[2], v.us[3]);
    std::fclose(f);
}

struct Events {
    cudaEvent_t e[kKernelsPerStep + 1] = {};
    bool ok = true;
    Events() {
        for (auto& x : e) ok = ok && cudaEventCreate(&x) == cudaSuccess;
    }
    ~Events() {
        for (auto& x : e)
            if (x) cudaEventDestroy(x);
    }
};

// One step of g with every kernel bracketed by events; adds the per-kernel times (ms).
template <typename T>
cudaError_t timed_step(const Dev& g, cudaStream_t s, Events& ev, float* ms) {
    cudaError_t e = cudaEventRecord(ev.e[0], s);
    for (int ph = 0; ph < kKernelsPerStep && e == cudaSuccess; ++ph) {
        launch_phase<T>(g, ph, s);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(ev.e[ph + 1], s);
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(ev.e[kKernelsPerStep]);
    for (int ph = 0; ph < kKernelsPerStep && e == cudaSuccess; ++ph)
        e = cudaEventElapsedTime(&ms[ph], ev.e[ph], ev.e[ph + 1]);
    return e;
}

// scalars for timing: buffer 0 current, budgets open (gated groups run every instance)
cudaError_t reset_scalars(const Dev& d, long long steps_left, cudaStream_t s) {
    std::vector<fdm_dev_scalars> h((size_t)d.count);
    std::memset(h.data(), 0, h.size() * sizeof(fdm_dev_scalars));
    for (auto& x : h) x.steps_left = steps_left;
    cudaError_t e = cudaMemcpyAsync(d.sc, h.data(), h.size() * sizeof(fdm_dev_scalars), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

}  // namespace

template <typename T>
cudaError_t autotune_group(Dev& d, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const fdm_params& p = d.p;
    const TuneKey key{dev, prec_code<T>(), p.n1, p.n2, d.count, d.gated, p.time_level, p.velocity_mode,
                      p.tau_y != 0.0 ? 1 : 0};
    int Rs[8], Cs[8];
    const int nR = row_candidates<T>(p.n1, p.n2, Rs, 8), nC = col_candidates<T>(p.n1, p.n2, Cs, 8);
    if (nR == 0 || nC == 0) return cudaSuccess;  // keep the heuristic shapes
    FileKey fkey;
    const bool have_id = device_identity(dev, &fkey.gpu, &fkey.sms);
    fkey.prec = prec_code<T>();
    fkey.n1 = p.n1;
    fkey.n2 = p.n2;
    fkey.count = d.count;
    fkey.gated = d.gated;
    fkey.tl = p.time_level;
    fkey.vm = p.velocity_mode;
    fkey.fr = p.tau_y != 0.0 ? 1 : 0;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            d.geom = it->second;
            return cudaSuccess;
        }
        load_file_cache();
        auto ft = have_id ? g_file_cache.find(fkey) : g_file_cache.end();
        if (ft != g_file_cache.end()) {
            const FileVal& v = ft->second;
            const bool r_ok = std::find(Rs, Rs + nR, v.R) != Rs + nR, c_ok = std::find(Cs, Cs + nC, v.C) != Cs + nC;
            if (r_ok && c_ok && v.shape >= 0 && v.shape < kKnpShapes) {
                LaunchGeom gm = geometry<T>(p.n1, p.n2, v.R, v.C, v.shape);
                gm.tuned = 1;
                for (int ph = 0; ph < kKernelsPerStep; ++ph) gm.kernel_us[ph] = v.us[ph];
                g_tune_cache.emplace(key, gm);
                d.geom = gm;
                return cudaSuccess;
            }
        }
    }
    Events ev;
    if (!ev.ok) return cudaErrorUnknown;
    launch_tune_fill<T>(d, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = reset_scalars(d, 1ll << 40, s)) != cudaSuccess) return e;

    const float kInf = 3.0e38f;
    std::vector<float> bestR(nR, kInf), bestC(nC, kInf), bestK(kKnpShapes, kInf);
    const int ncand = std::max(std::max(nR, nC), kKnpShapes);  // as fdm_launch_candidates
    constexpr int kReps = 3;
    Dev g = d;
    g.geom = geometry<T>(p.n1, p.n2);
    float ms[kKernelsPerStep];
    if ((e = timed_step<T>(g, s, ev, ms)) != cudaSuccess) return e;  // warm-up
    for (int i = 0; i < ncand; ++i) {
        const int ir = i % nR, ic = i % nC, ik = i % kKnpShapes;
        g.geom = geometry<T>(p.n1, p.n2, Rs[ir], Cs[ic], ik);
        if ((e = timed_step<T>(g, s, ev, ms)) != cudaSuccess) return e;  // first use of the shapes
        float best[kKernelsPerStep] = {kInf, kInf, kInf, kInf};
        for (int r = 0; r < kReps; ++r) {
            if ((e = timed_step<T>(g, s, ev, ms)) != cudaSuccess) return e;
            for (int ph = 0; ph < kKernelsPerStep; ++ph) best[ph] = std::min(best[ph], ms[ph]);
        }
        bestR[ir] = std::min(bestR[ir], best[0] + best[2]);
        bestC[ic] = std::min(bestC[ic], best[1]);
        bestK[ik] = std::min(bestK[ik], best[3]);
    }
    const int jr = (int)(std::min_element(bestR.begin(), bestR.end()) - bestR.begin());
    const int jc = (int)(std::min_element(bestC.begin(), bestC.end()) - bestC.begin());
    const int jk = (int)(std::min_element(bestK.begin(), bestK.end()) - bestK.begin());
    LaunchGeom best = geometry<T>(p.n1, p.n2, Rs[jr], Cs[jc], jk);
    // the kernels' times with the chosen shapes together
    float sum[kKernelsPerStep] = {kInf, kInf, kInf, kInf};
    g.geom = best;
    for (int r = 0; r < kReps; ++r) {
        if ((e = timed_step<T>(g, s, ev, ms)) != cudaSuccess) return e;
        for (int ph = 0; ph < kKernelsPerStep; ++ph) sum[ph] = std::min(sum[ph], ms[ph]);
    }
    best.tuned = 1;
    for (int ph = 0; ph < kKernelsPerStep; ++ph) best.kernel_us[ph] = 1000.0 * (double)sum[ph];
    if ((e = reset_scalars(d, 0, s)) != cudaSuccess) return e;
    d.geom = best;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache.emplace(key, best);
    if (have_id) {
        FileVal v{best.R, best.C, best.knp_shape, {}};
        for (int ph = 0; ph < kKernelsPerStep; ++ph) v.us[ph] = best.kernel_us[ph];
        g_file_cache[fkey] = v;
        append_file_cache(fkey, v);
    }
    return cudaSuccess;
}

template cudaError_t autotune_group<double>(Dev&, cudaStream_t);
template cudaError_t autotune_group<float>(Dev&, cudaStream_t);
template cudaError_t autotune_group<df>(Dev&, cudaStream_t);

}  // namespace fdm
