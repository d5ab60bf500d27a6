// fdm_batch.cu -- C ABI for batches of independent FDM instances (include/fdm.h):
// grouping by parameters, per-instance state upload/readout, step budgets, batched steps
// replayed from CUDA graphs.
#include <cstring>
#include <new>
#include <vector>

#include "fdm_df.cuh"
#include "fdm_host.h"

using namespace fdm;

struct fdm_batch {
    struct Group {
        Dev d;
        int prec;
        std::vector<int> members;      // batch indices of the group's instances
        std::vector<double> phi_ref;   // per instance (mixed precision offset)
    };
    std::vector<Group> groups;
    std::vector<int> group_of, local_of;
    Arena arena;
    StepGraphs graphs;
    cudaStream_t stream = nullptr;
    int count = 0;
    std::vector<bool> has_state;
    // persistent step (fdm_batch_enqueue_steps_persistent): group descriptors and the barrier
    void* persist_desc = nullptr;
    PersistBarrier* persist_bar = nullptr;
    size_t persist_smem = 0;
    bool persist_used = false;
};

namespace fdm {
// test hook of the persistent step's barrier (fdm_debug_barrier): arrivals expected beyond
// the grid, and the wait limit in seconds
int g_barrier_extra = 0;
double g_barrier_limit_s = 1.0;
}

namespace {

fdm_params resolved(const fdm_params& p) {
    fdm_params q = p;
    if (q.nz == 0) q.nz = q.n1;
    return q;
}

bool same_params(const fdm_params& a, const fdm_params& b) {
    return a.n1 == b.n1 && a.n2 == b.n2 && a.nz == b.nz && a.nh == b.nh && a.dx == b.dx && a.E == b.E &&
           a.nu == b.nu && a.velocity_mode == b.velocity_mode && a.v0 == b.v0 && a.mobility == b.mobility &&
           a.tau_y == b.tau_y && a.beta == b.beta && a.theta == b.theta && a.cfl == b.cfl &&
           a.dt_max == b.dt_max && a.loading_mode == b.loading_mode && a.sigma_bar13 == b.sigma_bar13 &&
           a.eps_bar13_0 == b.eps_bar13_0 && a.eps_bar13_rate == b.eps_bar13_rate &&
           a.time_level == b.time_level && a.precision == b.precision && a.autotune == b.autotune;
}

bool index_ok(const fdm_batch* b, int32_t i) { return b && i >= 0 && i < b->count; }

}  // namespace

extern "C" {

size_t fdm_batch_device_bytes(int32_t count, const fdm_params* params) {
    if (count < 1 || !params) return 0;
    size_t total = 0;
    for (int32_t i = 0; i < count; ++i) {
        size_t b = fdm_device_bytes(&params[i]);
        if (b == 0) return 0;
        total += b;
    }
    return total;
}

fdm_status fdm_batch_create(int32_t count, const fdm_params* params, void* stream, fdm_batch** out) {
    if (!out) return FDM_ERR_INVALID_ARG;
    *out = nullptr;
    if (count < 1 || !params) return FDM_ERR_INVALID_ARG;
    for (int32_t i = 0; i < count; ++i)
        if (!params_valid(&params[i])) return FDM_ERR_INVALID_ARG;
    fdm_batch* b = new (std::nothrow) fdm_batch();
    if (!b) return FDM_ERR_OOM;
    b->stream = (cudaStream_t)stream;
    b->count = count;
    b->group_of.assign(count, -1);
    b->local_of.assign(count, -1);
    b->has_state.assign(count, false);
    std::vector<fdm_params> keys;
    for (int32_t i = 0; i < count; ++i) {
        fdm_params q = resolved(params[i]);
        int g = -1;
        for (size_t k = 0; k < keys.size(); ++k)
            if (same_params(keys[k], q)) { g = (int)k; break; }
        if (g < 0) {
            keys.push_back(q);
            b->groups.emplace_back();
            g = (int)keys.size() - 1;
            b->groups[g].prec = q.precision;
        }
        b->group_of[i] = g;
        b->local_of[i] = (int)b->groups[g].members.size();
        b->groups[g].members.push_back(i);
    }
    for (size_t g = 0; g < b->groups.size(); ++g) {
        auto& G = b->groups[g];
        const int c = (int)G.members.size();
        fdm_status st = FDM_OK;
        FDM_DISPATCH(G.prec, st = build_group<T>(G.d, b->arena, keys[g], c, 1, false, b->stream));
        if (st != FDM_OK) {
            fdm_batch_destroy(b);
            return st;
        }
        G.phi_ref.assign(c, 0.0);
    }
    *out = b;
    return FDM_OK;
}

fdm_status fdm_batch_set_plastic_distortion(fdm_batch* b, int32_t i, const double* up13) {
    if (!index_ok(b, i) || !up13) return FDM_ERR_INVALID_ARG;
    auto& G = b->groups[b->group_of[i]];
    const int j = b->local_of[i];
    const size_t n = (size_t)G.d.p.n1 * G.d.p.n2;
    double mean = ksum(up13, n) / (double)n;
    if (!std::isfinite(mean)) return FDM_ERR_INVALID_ARG;
    FDM_CK(cudaStreamSynchronize(b->stream));
    const double ref = G.prec != FDM_FP64 ? mean : 0.0;
    fdm_status st = upload_state(G.d, G.prec, 0, j, up13, ref, b->stream);
    if (st) return st;
    fdm_dev_scalars s;
    std::memset(&s, 0, sizeof(s));
    s.phi_ref = ref;
    s.mean_up13 = mean;
    s.cur = 0;
    s.steps_left = 0;
    host_loading(G.d.p, 0, 0.0, mean, &s.eps_bar13, &s.sigma_bar13);
    FDM_CK(cudaMemcpyAsync(G.d.sc + j, &s, sizeof(s), cudaMemcpyHostToDevice, b->stream));
    FDM_CK(cudaStreamSynchronize(b->stream));
    G.phi_ref[j] = ref;
    b->has_state[i] = true;
    return FDM_OK;
}

fdm_status fdm_batch_set_budget(fdm_batch* b, int32_t i, int64_t steps) {
    if (!index_ok(b, i) || steps < 0) return FDM_ERR_INVALID_ARG;
    if (!b->has_state[i]) return FDM_ERR_STATE;
    auto& G = b->groups[b->group_of[i]];
    const int j = b->local_of[i];
    static_assert(sizeof(long long) == sizeof(int64_t), "budget width");
    // pageable source: the copy completes before the call returns
    long long v = (long long)steps;
    FDM_CK(cudaMemcpyAsync(&G.d.sc[j].steps_left, &v, sizeof(v), cudaMemcpyHostToDevice, b->stream));
    FDM_CK(cudaStreamSynchronize(b->stream));
    return FDM_OK;
}

fdm_status fdm_batch_enqueue_steps(fdm_batch* b, int32_t nsteps) {
    if (!b || nsteps < 0) return FDM_ERR_INVALID_ARG;
    if (nsteps == 0) return FDM_OK;
    std::vector<Dev*> devs;
    std::vector<int> prec;
    for (auto& G : b->groups) {
        devs.push_back(&G.d);
        prec.push_back(G.prec);
    }
    fdm_status st = build_step_graphs(b->graphs, devs, prec);
    if (st) return st;
    return replay_steps(b->graphs, nsteps, b->stream);
}

// FDM_ERR_TIMEOUT if the last persistent launch of the batch gave up at a barrier (waits);
// the status is reported once
static fdm_status persist_status(fdm_batch* b) {
    if (!b->persist_used) return FDM_OK;
    int st = 0;
    FDM_CK(cudaMemcpyAsync(&st, &b->persist_bar->status, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    FDM_CK(cudaStreamSynchronize(b->stream));
    b->persist_used = false;
    return (fdm_status)st;
}

fdm_status fdm_batch_enqueue_steps_persistent(fdm_batch* b, int32_t nsteps) {
    if (!b || nsteps < 0) return FDM_ERR_INVALID_ARG;
    if (nsteps == 0) return FDM_OK;
    const int ng = (int)b->groups.size();
    std::vector<const Dev*> devs;
    for (auto& G : b->groups) devs.push_back(&G.d);
    fdm_status st;
    if (!b->persist_desc) {
        std::vector<unsigned char> host(persist_group_bytes() * ng);
        size_t smem = 0;
        if ((st = persist_prepare(devs.data(), ng, host.data(), &smem))) return st;
        void* desc = nullptr;
        void* bar = nullptr;
        if ((st = b->arena.alloc(&desc, host.size()))) return st;
        if ((st = b->arena.alloc(&bar, sizeof(PersistBarrier)))) return st;
        FDM_CK(cudaMemcpyAsync(desc, host.data(), host.size(), cudaMemcpyHostToDevice, b->stream));
        FDM_CK(cudaStreamSynchronize(b->stream));
        b->persist_desc = desc;
        b->persist_bar = (PersistBarrier*)bar;
        b->persist_smem = smem;
    }
    // a fresh barrier for this launch
    int dev = 0, khz = 0;
    FDM_CK(cudaGetDevice(&dev));
    FDM_CK(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    PersistBarrier pb;
    std::memset(&pb, 0, sizeof(pb));
    pb.extra = g_barrier_extra;
    pb.limit_cycles = (long long)(g_barrier_limit_s * (double)khz * 1e3);
    FDM_CK(cudaMemcpyAsync(b->persist_bar, &pb, sizeof(pb), cudaMemcpyHostToDevice, b->stream));
    FDM_CK(cudaStreamSynchronize(b->stream));
    FDM_CK(persist_launch(b->persist_desc, ng, nsteps, b->persist_bar, b->persist_smem, b->stream));
    b->persist_used = true;
    return FDM_OK;
}

void fdm_debug_barrier(int32_t extra_arrivals, double limit_seconds) {
    g_barrier_extra = extra_arrivals > 0 ? extra_arrivals : 0;
    g_barrier_limit_s = limit_seconds > 0.0 ? limit_seconds : 1.0;
}

fdm_status fdm_batch_sync(fdm_batch* b, int64_t* steps_left) {
    if (!b) return FDM_ERR_INVALID_ARG;
    fdm_status first = persist_status(b);
    for (auto& G : b->groups) {
        std::vector<fdm_dev_scalars> s(G.members.size());
        FDM_CK(cudaMemcpyAsync(s.data(), G.d.sc, s.size() * sizeof(fdm_dev_scalars), cudaMemcpyDeviceToHost,
                               b->stream));
        FDM_CK(cudaStreamSynchronize(b->stream));
        for (size_t j = 0; j < s.size(); ++j) {
            if (steps_left) steps_left[G.members[j]] = (int64_t)s[j].steps_left;
            if (s[j].status && first == FDM_OK) first = (fdm_status)s[j].status;
        }
    }
    return first;
}

fdm_status fdm_batch_sync_status(fdm_batch* b, int64_t* steps_left, int32_t* status) {
    if (!b) return FDM_ERR_INVALID_ARG;
    if (fdm_status pst = persist_status(b)) return pst;
    for (auto& G : b->groups) {
        std::vector<fdm_dev_scalars> s(G.members.size());
        FDM_CK(cudaMemcpyAsync(s.data(), G.d.sc, s.size() * sizeof(fdm_dev_scalars), cudaMemcpyDeviceToHost,
                               b->stream));
        FDM_CK(cudaStreamSynchronize(b->stream));
        for (size_t j = 0; j < s.size(); ++j) {
            if (steps_left) steps_left[G.members[j]] = (int64_t)s[j].steps_left;
            if (status) status[G.members[j]] = (int32_t)s[j].status;
        }
    }
    return FDM_OK;
}

fdm_status fdm_batch_get_info(fdm_batch* b, int32_t i, fdm_step_info* info) {
    if (!index_ok(b, i) || !info) return FDM_ERR_INVALID_ARG;
    if (!b->has_state[i]) return FDM_ERR_STATE;
    auto& G = b->groups[b->group_of[i]];
    return instance_info(G.d, b->local_of[i], G.prec, b->stream, info);
}

fdm_status fdm_batch_read_fields(fdm_batch* b, int32_t i, uint32_t mask, double* up13, double* tau13) {
    if (!index_ok(b, i)) return FDM_ERR_INVALID_ARG;
    if (mask & ~(uint32_t)(FDM_FIELD_UP13 | FDM_FIELD_TAU13)) return FDM_ERR_INVALID_ARG;
    if (((mask & FDM_FIELD_UP13) && !up13) || ((mask & FDM_FIELD_TAU13) && !tau13)) return FDM_ERR_INVALID_ARG;
    if (!b->has_state[i]) return FDM_ERR_STATE;
    auto& G = b->groups[b->group_of[i]];
    const int j = b->local_of[i];
    const size_t n = (size_t)G.d.p.n1 * G.d.p.n2;
    const size_t e = elt_size(&G.d.p);
    fdm_dev_scalars s;
    FDM_CK(cudaMemcpyAsync(&s, G.d.sc + j, sizeof(s), cudaMemcpyDeviceToHost, b->stream));
    FDM_CK(cudaStreamSynchronize(b->stream));
    fdm_status st;
    if (mask & FDM_FIELD_UP13)
        if ((st = download_state(up13, G.d, G.prec, s.cur, j, G.phi_ref[j], b->stream))) return st;
    if (mask & FDM_FIELD_TAU13)
        if ((st = download_field(tau13, (char*)G.d.tau + (size_t)j * n * e, n, G.prec, 0.0, b->stream)))
            return st;
    return FDM_OK;
}

int32_t fdm_batch_launches_per_step(const fdm_batch* b) {
    return b ? (int32_t)(kKernelsPerStep * b->groups.size()) : 0;
}

fdm_status fdm_batch_get_launch_config(const fdm_batch* b, int32_t i, fdm_launch_config* cfg) {
    if (!index_ok(b, i) || !cfg) return FDM_ERR_INVALID_ARG;
    const fdm_batch::Group& G = b->groups[b->group_of[i]];
    FDM_DISPATCH(G.prec, launch_config<T>(G.d.geom, cfg));
    return FDM_OK;
}

void fdm_batch_destroy(fdm_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    b->graphs.destroy();
    b->arena.free_all();
    delete b;
}

}  // extern "C"
