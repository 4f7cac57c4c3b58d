// tune.cu -- one persistent launch for all models of a handle, and the launch-shape autotuner.
//
// Batching environments of different skeletons: instead of one step launch per model (each with
// its own tail of idle SMs), k_step_mixed takes work items of every model from one queue.  The
// autotuner times the candidate launch shapes (warps per environment, environments per block,
// whether the via points are staged in shared memory) of the per-model launches and of the
// mixed launch on the handle's own environments, keeps the fastest, and can cache the choice in
// a text file keyed by the models, the environment counts, the device and the substep count.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "handle.h"

using namespace msim;
using namespace msim::host;

namespace {

// rough cost of one environment-substep, to order the queue (expensive models first)
long long model_cost(const ImgHeader& h) {
    return 4LL * h.n_packed + 8LL * h.nnz + 10LL * h.m + 30LL * h.nb;
}

int slots_limit(int wpe) { return wpe == 1 ? 16 : std::min(15, 16 / wpe); }

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
    const uint8_t* b = static_cast<const uint8_t*>(p);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

uint64_t tune_key(msim_handle h, int n_sub) {
    uint64_t k = 1469598103934665603ull;
    for (int i = 0; i < h->n_models; ++i) {
        const std::vector<uint8_t>& b = h->models[i].blob;
        k = fnv1a(k, b.data(), b.size());
        const int ne = h->env_begin[i + 1] - h->env_begin[i];
        k = fnv1a(k, &ne, sizeof(ne));
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, h->device) == cudaSuccess) {
        k = fnv1a(k, prop.name, std::strlen(prop.name));
        k = fnv1a(k, &prop.multiProcessorCount, sizeof(int));
    }
    k = fnv1a(k, &n_sub, sizeof(n_sub));
    const int version = msim_version();
    return fnv1a(k, &version, sizeof(version));
}

}  // namespace

namespace msim {
namespace host {

// Staging levels of a mixed launch from a mask: bit i = model i fully staged (level 1); else
// bit 8 + i = its muscle records also read through the cache (level 2); else level 0.
void mask_levels(int32_t mask, int* lv) {
    for (int i = 0; i < kMaxModels; ++i) lv[i] = ((mask >> i) & 1) ? 1 : (((mask >> (8 + i)) & 1) ? 2 : 0);
}
int32_t levels_mask(const int* lv, int n) {
    int32_t m = 0;
    for (int i = 0; i < n; ++i) m |= lv[i] == 1 ? (1 << i) : (lv[i] == 2 ? (1 << (8 + i)) : 0);
    return m;
}

bool mixed_args(msim_handle h, int wpe, int slots, const int* pts, MixedArgs* out, size_t* smem, int* grid) {
    if (wpe != 1 && wpe != 2 && wpe != 4) return false;
    if (slots < 1 || slots > slots_limit(wpe)) return false;
    MixedArgs m;
    std::memset(&m, 0, sizeof(m));
    int order[kMaxModels], no = 0;
    for (int i = 0; i < h->n_models; ++i)
        if (h->env_begin[i + 1] > h->env_begin[i]) order[no++] = i;
    if (no == 0) return false;
    std::stable_sort(order, order + no,
                     [&](int a, int b) { return model_cost(h->models[a].hdr) > model_cost(h->models[b].hdr); });
    size_t region = 0;
    for (int k = 0; k < no; ++k) {
        const ImgHeader& hd = h->models[order[k]].hdr;
        const size_t staged = (size_t)staged_bytes(hd, pts[order[k]]);
        region = std::max(region, (staged + 127) & ~(size_t)127);
    }
    if (16 + region >= h->smem_optin) return false;
    const size_t avail = h->smem_optin - 16 - region;
    size_t ws_max = 0;
    int items = 0;
    for (int k = 0; k < no; ++k) {
        const int i = order[k];
        const ImgHeader& hd = h->models[i].hdr;
        const size_t per = (size_t)ws_floats(hd, wpe) * sizeof(float);
        const int ne = h->env_begin[i + 1] - h->env_begin[i];
        const int epb = (int)std::min<size_t>({(size_t)slots, avail / per, (size_t)ne});
        if (epb < 1) return false;
        MixedModel& M = m.mdl[k];
        M.img = h->d_img[i];
        M.stage = pts[i];
        M.staged_bytes = staged_bytes(hd, M.stage);
        M.env_begin = h->env_begin[i];
        M.env_end = h->env_begin[i + 1];
        M.epb = epb;
        M.item_begin = items;
        items += (ne + epb - 1) / epb;
        ws_max = std::max(ws_max, (size_t)epb * per);
    }
    m.a = base_args(h, order[0]);
    m.a.wpe = wpe;
    m.n_models = no;
    m.n_items = items;
    m.slots = slots;
    m.img_region = (int)region;
    m.queue = h->queue;
    const size_t sm = 16 + region + ws_max;
    if (sm > h->smem_optin) return false;
    for (int k = 0; k < no; ++k) m.wrap |= uses_ext(h->models[order[k]].hdr) ? 1 : 0;
    const int per_sm = mixed_blocks_per_sm(32 * wpe * slots, sm, wpe, m.wrap != 0);
    if (per_sm < 1) return false;
    *out = m;
    *smem = sm;
    *grid = std::max(1, std::min(items, h->num_sms * per_sm));
    return true;
}

cudaError_t launch_all(msim_handle h, const float* exc, int n_sub, cudaStream_t s) {
    if (h->mixed) {
        MixedArgs m;
        size_t smem = 0;
        int grid = 0;
        if (!mixed_args(h, h->mixed_wpe, h->mixed_slots, h->mixed_pts, &m, &smem, &grid)) return cudaErrorInvalidValue;
        m.a.exc = exc;
        m.a.n_sub = n_sub;
        return launch_mixed(m, grid, smem, s);
    }
    for (int i = 0; i < h->n_models; ++i) {
        if (h->env_begin[i + 1] == h->env_begin[i]) continue;
        StepArgs a = base_args(h, i);
        a.exc = exc;
        a.n_sub = n_sub;
        const cudaError_t e =
            launch_step(a, model_grid(h, i), step_smem_bytes(h->models[i].hdr, h->epb[i], h->pts_smem[i], h->wpe[i]), s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace host
}  // namespace msim

namespace {

// Saves the handle's state buffers so that timed launches leave no trace.
struct Snapshot {
    float *q = nullptr, *qd = nullptr, *act = nullptr, *qdd = nullptr, *force = nullptr, *eps = nullptr,
          *vm = nullptr;
    uint32_t *st = nullptr, *gf = nullptr;
    size_t rn = 0, rm = 0, ne = 0;
    cudaError_t take(msim_handle h, cudaStream_t s) {
        rn = (size_t)h->n_envs * h->pitch_n * 4;
        rm = (size_t)h->n_envs * h->pitch_m * 4;
        ne = (size_t)h->n_envs * 4;
        cudaError_t e = cudaMalloc(&q, rn);
        if (e == cudaSuccess) e = cudaMalloc(&qd, rn);
        if (e == cudaSuccess) e = cudaMalloc(&qdd, rn);
        if (e == cudaSuccess) e = cudaMalloc(&act, rm);
        if (e == cudaSuccess) e = cudaMalloc(&force, rm);
        if (e == cudaSuccess) e = cudaMalloc(&eps, rm);
        if (e == cudaSuccess && h->vm) e = cudaMalloc(&vm, rm);
        if (e == cudaSuccess) e = cudaMalloc(&st, ne);
        if (e == cudaSuccess) e = cudaMalloc(&gf, 4);
        if (e == cudaSuccess) e = copy(h, true, s);
        return e;
    }
    cudaError_t copy(msim_handle h, bool save, cudaStream_t s) {
        auto cp = [&](void* a, void* b, size_t n) {
            return cudaMemcpyAsync(save ? a : b, save ? b : a, n, cudaMemcpyDeviceToDevice, s);
        };
        cudaError_t e = cp(q, h->q, rn);
        if (e == cudaSuccess) e = cp(qd, h->qd, rn);
        if (e == cudaSuccess) e = cp(qdd, h->qdd, rn);
        if (e == cudaSuccess) e = cp(act, h->act, rm);
        if (e == cudaSuccess) e = cp(force, h->force, rm);
        if (e == cudaSuccess) e = cp(eps, h->eps, rm);   // tendon strains: state like q and act
        if (e == cudaSuccess && vm) e = cp(vm, h->vm, rm);
        if (e == cudaSuccess) e = cp(st, h->env_status, ne);
        if (e == cudaSuccess) e = cp(gf, h->gflags, 4);
        return e;
    }
    ~Snapshot() {
        cudaFree(q); cudaFree(qd); cudaFree(qdd); cudaFree(act); cudaFree(force); cudaFree(eps); cudaFree(vm);
        cudaFree(st); cudaFree(gf);
    }
};

bool read_cache(const char* path, uint64_t key, msim_tune_result* r) {
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        unsigned long long k = 0;
        int off = 0;
        if (std::sscanf(line, "msim-tune-v1 %llx%n", &k, &off) != 1 || k != key) continue;
        msim_tune_result t;
        std::memset(&t, 0, sizeof(t));
        int n = 0, used = 0;
        const char* p = line + off;
        if (std::sscanf(p, " %d %d %d %d %d%n", &t.mixed, &t.mixed_warps_per_env, &t.mixed_slots,
                        &t.mixed_stage_points_mask, &n, &used) != 5 || n < 1 || n > kMaxModels)
            continue;
        p += used;
        bool ok = true;
        for (int i = 0; i < n && ok; ++i) {
            ok = std::sscanf(p, " %d %d %d%n", &t.warps_per_env[i], &t.envs_per_block[i], &t.stage_points[i], &used) == 3;
            p += used;
        }
        if (!ok || std::sscanf(p, " %f %f", &t.ms_per_model, &t.ms_mixed) != 2) continue;
        *r = t;
        found = true;   // the last matching line wins
    }
    std::fclose(f);
    return found;
}

void write_cache(const char* path, uint64_t key, int n_models, const msim_tune_result& t) {
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "msim-tune-v1 %016llx %d %d %d %d %d", (unsigned long long)key, t.mixed, t.mixed_warps_per_env,
                 t.mixed_slots, t.mixed_stage_points_mask, n_models);
    for (int i = 0; i < n_models; ++i)
        std::fprintf(f, " %d %d %d", t.warps_per_env[i], t.envs_per_block[i], t.stage_points[i]);
    std::fprintf(f, " %.6f %.6f\n", t.ms_per_model, t.ms_mixed);
    std::fclose(f);
}

// applies a result; false if a shape no longer fits (the cache then is ignored)
bool apply(msim_handle h, const msim_tune_result& t) {
    for (int i = 0; i < h->n_models; ++i) {
        const int w = t.warps_per_env[i], e = t.envs_per_block[i];
        const int p = t.stage_points[i];
        if ((w != 1 && w != 2 && w != 4) || p < 0 || p > 2 || e < 1 || e > max_epb(h, i, p, w)) return false;
    }
    int pts[kMaxModels];
    mask_levels(t.mixed_stage_points_mask, pts);
    if (t.mixed) {
        MixedArgs m;
        size_t sm;
        int grid;
        if (!mixed_args(h, t.mixed_warps_per_env, t.mixed_slots, pts, &m, &sm, &grid)) return false;
    }
    for (int i = 0; i < h->n_models; ++i) {
        h->wpe[i] = t.warps_per_env[i];
        h->epb[i] = t.envs_per_block[i];
        h->pts_smem[i] = t.stage_points[i];
    }
    h->mixed = t.mixed ? 1 : 0;
    h->mixed_wpe = t.mixed_warps_per_env;
    h->mixed_slots = t.mixed_slots;
    for (int i = 0; i < kMaxModels; ++i) h->mixed_pts[i] = pts[i];
    return true;
}

}  // namespace

extern "C" {

msim_status msim_set_mixed_launch(msim_handle h, int32_t enable, int32_t warps_per_env, int32_t slots_per_block,
                                  int32_t stage_points_mask) {
    if (!h) return arg_fail(h, "msim_set_mixed_launch: NULL handle");
    if (!enable) {
        h->mixed = 0;
        return MSIM_OK;
    }
    const int w = warps_per_env == 0 ? 2 : warps_per_env;
    int pts[kMaxModels];
    if (stage_points_mask < 0) {
        for (int i = 0; i < kMaxModels; ++i) pts[i] = h->pts_smem[i];
    } else {
        mask_levels(stage_points_mask, pts);
    }
    MixedArgs m;
    size_t sm;
    int grid;
    int slots = slots_per_block;
    if (slots == 0) {   // largest that fits, at most 8
        for (slots = std::min(8, slots_limit(w)); slots >= 1; --slots)
            if (mixed_args(h, w, slots, pts, &m, &sm, &grid)) break;
    }
    if (slots < 1 || !mixed_args(h, w, slots, pts, &m, &sm, &grid))
        return arg_fail(h, "msim_set_mixed_launch: shape does not fit (threads, barriers or shared memory)");
    h->mixed = 1;
    h->mixed_wpe = w;
    h->mixed_slots = slots;
    for (int i = 0; i < kMaxModels; ++i) h->mixed_pts[i] = pts[i];
    return MSIM_OK;
}

msim_status msim_autotune(msim_handle h, const char* cache_path, int32_t n_substeps, msim_tune_result* out) {
    if (!h) return arg_fail(h, "msim_autotune: NULL handle");
    if (n_substeps < 1 || n_substeps > 1000) return arg_fail(h, "msim_autotune: n_substeps must be 1..1000");
    msim_tune_result r;
    std::memset(&r, 0, sizeof(r));
    cudaSetDevice(h->device);
    const uint64_t key = tune_key(h, n_substeps);
    if (cache_path && read_cache(cache_path, key, &r) && apply(h, r)) {
        r.from_cache = 1;
        if (out) *out = r;
        return MSIM_OK;
    }
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    Snapshot snap;
    if (e == cudaSuccess) e = snap.take(h, s);
    const size_t rm = (size_t)h->n_envs * h->pitch_m * 4;
    if (e == cudaSuccess) e = cudaMemsetAsync(h->exc_stage, 0, rm, s);   // excitation 0 while timing
    if (e != cudaSuccess) {
        if (s) cudaStreamDestroy(s);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        return cuda_fail(h, e, "msim_autotune setup");
    }
    int candidates = 0;
    // time one configuration: restore, warm launch, restore, timed launch; best of two timed
    auto timed = [&](auto&& launch) -> float {
        float best = 1e30f;
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
            e = snap.copy(h, false, s);
            if (e == cudaSuccess) e = cudaEventRecord(e0, s);
            if (e == cudaSuccess) e = launch();
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && rep > 0) best = std::min(best, ms);
        }
        ++candidates;
        return best;
    };
    const int epb_cands[] = {1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 14, 16};
    // 1. per-model launches, each model on its own
    for (int i = 0; i < h->n_models && e == cudaSuccess; ++i) {
        const int ne = h->env_begin[i + 1] - h->env_begin[i];
        r.warps_per_env[i] = h->wpe[i];
        r.envs_per_block[i] = h->epb[i];
        r.stage_points[i] = h->pts_smem[i];
        if (ne == 0) continue;
        float best = 1e30f;
        for (int w : {1, 2, 4}) {
            for (int p = 0; p <= 2; ++p) {
                const int emax = std::min(max_epb(h, i, p, w), ne);
                for (int ep : epb_cands) {
                    if (ep > emax || e != cudaSuccess) continue;
                    h->wpe[i] = w; h->epb[i] = ep; h->pts_smem[i] = p;
                    StepArgs a = base_args(h, i);
                    a.exc = h->exc_stage;
                    a.n_sub = n_substeps;
                    const int grid = model_grid(h, i);
                    const size_t sm = step_smem_bytes(h->models[i].hdr, ep, p, w);
                    const float t = timed([&]() { return launch_step(a, grid, sm, s); });
                    if (t < best) {
                        best = t;
                        r.warps_per_env[i] = w; r.envs_per_block[i] = ep; r.stage_points[i] = p;
                    }
                }
            }
        }
        h->wpe[i] = r.warps_per_env[i]; h->epb[i] = r.envs_per_block[i]; h->pts_smem[i] = r.stage_points[i];
    }
    // 2. the per-model launches back to back, as msim_step issues them
    h->mixed = 0;
    if (e == cudaSuccess) r.ms_per_model = timed([&]() { return launch_all(h, h->exc_stage, n_substeps, s); });
    // 3. one mixed launch (only with environments of two or more models)
    float best_mixed = 1e30f;
    int best_w = 0, best_sl = 0, best_mask = 0;
    int mask_best = 0, populated = 0;
    for (int i = 0; i < h->n_models; ++i) populated += h->env_begin[i + 1] > h->env_begin[i];
    mask_best = levels_mask(r.stage_points, h->n_models);
    const int32_t all_cached = levels_mask(std::vector<int>(h->n_models, 2).data(), h->n_models);
    for (int w : {1, 2, 4}) {
        if (populated < 2) break;
        for (int sl = 1; sl <= slots_limit(w); ++sl) {
            const int32_t masks[3] = {mask_best, 0, all_cached};
            for (int mi = 0; mi < 3; ++mi) {
                const int32_t mask = masks[mi];
                if (e != cudaSuccess) break;
                if ((mi == 1 && mask == mask_best) || (mi == 2 && (mask == mask_best || mask == 0))) continue;
                int pts[kMaxModels];
                mask_levels(mask, pts);
                MixedArgs m;
                size_t sm;
                int grid;
                if (!mixed_args(h, w, sl, pts, &m, &sm, &grid)) continue;
                m.a.exc = h->exc_stage;
                m.a.n_sub = n_substeps;
                const float t = timed([&]() { return launch_mixed(m, grid, sm, s); });
                if (t < best_mixed) {
                    best_mixed = t;
                    best_w = w; best_sl = sl; best_mask = mask;
                }
            }
        }
    }
    cudaError_t e2 = snap.copy(h, false, s);   // leave the state as it was
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "msim_autotune");
    r.ms_mixed = best_w ? best_mixed : 0.f;
    r.mixed = (best_w && best_mixed < r.ms_per_model) ? 1 : 0;
    r.mixed_warps_per_env = best_w ? best_w : 2;
    r.mixed_slots = best_w ? best_sl : 4;
    r.mixed_stage_points_mask = best_w ? best_mask : mask_best;
    r.candidates = candidates;
    apply(h, r);
    if (cache_path) write_cache(cache_path, key, h->n_models, r);
    if (out) *out = r;
    return MSIM_OK;
}

}  // extern "C"
