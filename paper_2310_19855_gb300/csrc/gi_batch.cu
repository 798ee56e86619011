// Many views per frame: the whole pass chain (spawn, update, resolve, probe irradiance,
// interpolation) with one launch per pass over every view, optionally replayed from a CUDA graph.
//
// Each view keeps its own cache (gi_cache_t) and buffers.  Per frame the host writes every view's
// pass arguments and the per-pass prefix tables of block counts into a pinned descriptor buffer;
// one copy moves it to the device, then six launches run the passes over all views (a block
// finds its view by binary search in the prefix table).  In graph mode the copy and the launches
// are captured once per descriptor buffer (two buffers, alternating) and replayed every frame;
// compactions of a table, decided on the host, run before the replay, outside the graph.
//
// With surrogates (gi_batch_set_surrogate: one for every view; gi_batch_set_view_surrogates: one
// per view, or none), the update keeps the far-hit routing of the caches that route to their
// view's surrogate, and the probe-irradiance pass becomes, per view, the surrogate's query frame
// and the probe pass with its answers (gi_nrc_query_frame, gi_probes_integrate_nrc; a network's
// answer buffers hold one view's records at a time), on side streams beside one batched probe
// pass over the views without one.  That form runs without the graph.
#include <string.h>

#include <algorithm>
#include <vector>

#include "gi_internal.cuh"

namespace gi {

struct DescLayout {
    size_t upd, res, spawn, integ, interp, pre[5], total;
};

static size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

static DescLayout desc_layout(uint32_t n) {
    DescLayout L;
    size_t o = 0;
    L.upd = o; o = align16(o + n * sizeof(UpdateArgs));
    L.res = o; o = align16(o + n * sizeof(ResolveArgs));
    L.spawn = o; o = align16(o + n * sizeof(SpawnArgs));
    L.integ = o; o = align16(o + n * sizeof(IntegrateArgs));
    L.interp = o; o = align16(o + n * sizeof(InterpArgs));
    for (int k = 0; k < 5; ++k) {  // n + 1 prefix entries, then the pass's work-item counter
        L.pre[k] = o;
        o = align16(o + (n + 2) * sizeof(uint32_t));
    }
    L.total = o;
    return L;
}

enum { kPassSpawn = 0, kPassUpdate, kPassResolve, kPassIntegrate, kPassInterp };

} // namespace gi

struct gi_batch_s {
    uint32_t n, rpp;
    gi_batch_tuning tuning;
    int sms;
    gi::DescLayout L;
    unsigned char *d_desc;
    unsigned char *h_desc[2];
    cudaEvent_t used[2];
    bool used_recorded[2];
    int set;
    cudaGraphExec_t exec[2];
    std::vector<uint32_t> sig[2];  // block counts the graph of each buffer was captured with
    cudaStream_t capture;          // private stream the graphs are captured on
    uint64_t frames;
    std::vector<gi_nrc_t> nrcs;    // surrogate of each view's probe pass, or NULL
    bool surr;                     // some view has one: the probe pass runs per view
    // streams of the surrogate views' probe passes: distinct networks run side by side (a
    // network's answer buffers hold one view at a time, so views that share one share a stream)
    cudaStream_t side[4];
    cudaEvent_t fork, join[4];
};

namespace gi {

static bool tuning_ok(const gi_batch_tuning *t) {
    return t && t->update_records_per_block >= 256 && t->update_records_per_block <= 2048 &&
           t->update_records_per_block % 256 == 0 && t->resolve_blocks_per_sm >= 1 && t->resolve_blocks_per_sm <= 4 &&
           t->integrate_threads >= 32 && t->integrate_threads <= 128 && t->integrate_threads % 32 == 0;
}

static void drop_graphs(gi_batch_s *b) {
    for (int k = 0; k < 2; ++k) {
        if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
        b->exec[k] = nullptr;
        b->sig[k].clear();
    }
}

static void free_batch(gi_batch_s *b) {
    drop_graphs(b);
    cudaFree(b->d_desc);
    for (int k = 0; k < 2; ++k) {
        if (b->h_desc[k]) cudaFreeHost(b->h_desc[k]);
        if (b->used[k]) cudaEventDestroy(b->used[k]);
    }
    if (b->capture) cudaStreamDestroy(b->capture);
    for (int k = 0; k < 4; ++k) {
        if (b->side[k]) cudaStreamDestroy(b->side[k]);
        if (b->join[k]) cudaEventDestroy(b->join[k]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

static gi_status check_view(const gi_batch_view &v, uint32_t rpp, int key_dir) {
    if (!v.cache) {
        set_error("gi_batch_frame: a view has no cache");
        return GI_ERR_INVALID_ARG;
    }
    if (cache_tiled(v.cache)) {
        set_error("gi_batch_frame: tile caches run through the single-view calls");
        return GI_ERR_INVALID_ARG;
    }
    if (cache_key_dir(v.cache) != key_dir) {
        set_error("gi_batch_frame: every cache of a batch must use the same direction descriptor");
        return GI_ERR_INVALID_ARG;
    }
    if (!hits_ok(&v.hits, (uint32_t)key_dir) || !view_ok(&v.view) || !v.slot_ids) {
        set_error("gi_batch_frame: a view has a NULL record plane or slot-id buffer, or a bad view");
        return GI_ERR_INVALID_ARG;
    }
    gi_status s = spawn_check(&v.gbuf, &v.view, &v.probes);
    if (s == GI_OK) s = integrate_check(v.cache, &v.probes, v.slot_ids, rpp);
    if (s == GI_OK) s = interp_check(&v.gbuf, &v.view, &v.probes, v.irradiance);
    if (s != GI_OK) return s;
    if (v.hits.n != (uint64_t)v.probes.layout.num_probes * rpp) {
        set_error("gi_batch_frame: a view has %llu records, expected probes x rays_per_probe = %llu",
                  (unsigned long long)v.hits.n, (unsigned long long)v.probes.layout.num_probes * rpp);
        return GI_ERR_INVALID_ARG;
    }
    return GI_OK;
}

// Enqueue the descriptor copy and the six batched launches on st (with a surrogate, the probe
// pass per view: views must then be given).
static gi_status enqueue_frame(gi_batch_s *b, int set, const std::vector<uint32_t> &blocks, int key_dir,
                               cudaStream_t st, const gi_batch_view *views = nullptr) {
    const DescLayout &L = b->L;
    unsigned char *d = b->d_desc;
    gi_status s = cuda_status(cudaMemcpyAsync(d, b->h_desc[set], L.total, cudaMemcpyHostToDevice, st),
                              "batch descriptor copy");
    const uint32_t n = b->n;
    if (s == GI_OK)
        s = launch_spawn_batched(reinterpret_cast<const SpawnArgs *>(d + L.spawn),
                                 reinterpret_cast<const uint32_t *>(d + L.pre[kPassSpawn]), n, blocks[kPassSpawn], st);
    if (s == GI_OK)
        s = launch_update_batched(reinterpret_cast<const UpdateArgs *>(d + L.upd),
                                  reinterpret_cast<const uint32_t *>(d + L.pre[kPassUpdate]), n, blocks[kPassUpdate],
                                  key_dir, st);
    if (s == GI_OK)
        s = launch_resolve_batched(reinterpret_cast<const ResolveArgs *>(d + L.res),
                                   reinterpret_cast<const uint32_t *>(d + L.pre[kPassResolve]), n,
                                   blocks[kPassResolve], st);
    // the views with a surrogate: query frame and probe pass with its answers, per view, on the
    // side streams (from the resolve on), beside one launch over the views without one (all of
    // them in the plain form; a view with a surrogate has no blocks in it)
    const bool per_view = s == GI_OK && b->surr && views;
    gi_nrc_t owner[4] = {nullptr, nullptr, nullptr, nullptr};
    if (per_view) s = cuda_status(cudaEventRecord(b->fork, st), "fork record");
    if (s == GI_OK)
        s = launch_integrate_batched(reinterpret_cast<const IntegrateArgs *>(d + L.integ),
                                     reinterpret_cast<const uint32_t *>(d + L.pre[kPassIntegrate]), n,
                                     blocks[kPassIntegrate], b->tuning.integrate_threads, b->rpp, st);
    if (per_view) {
        int used = 0;
        for (uint32_t v = 0; v < n && s == GI_OK; ++v) {
            const gi_batch_view &bv = views[v];
            const gi_nrc_t nrc = b->nrcs[v];
            if (!nrc) continue;
            // the stream of this network: the one it already has, else the next (round robin)
            int k = 0;
            while (k < used && owner[k] != nrc) ++k;
            if (k == used) {
                if (used < 4) {
                    owner[used++] = nrc;
                    s = cuda_status(cudaStreamWaitEvent(b->side[k], b->fork, 0), "side stream wait");
                } else {
                    // more than four networks: the others share the streams, each network always
                    // on the same one (every side stream has waited for the fork by now)
                    k = (int)(((uintptr_t)nrc >> 6) % 4u);
                }
            }
            cudaStream_t ss = b->side[k];
            if (s == GI_OK) s = gi_nrc_query_frame(nrc, bv.cache, &bv.hits, bv.slot_ids, &bv.view, ss);
            if (s == GI_OK) s = gi_probes_integrate_nrc(bv.cache, nrc, &bv.probes, bv.slot_ids, b->rpp, bv.env, ss);
        }
        // the frame's later work waits for every side stream, also after an error above
        for (int k = 0; k < used; ++k) {
            gi_status sj = cuda_status(cudaEventRecord(b->join[k], b->side[k]), "join record");
            if (sj == GI_OK) sj = cuda_status(cudaStreamWaitEvent(st, b->join[k], 0), "join wait");
            if (s == GI_OK) s = sj;
        }
    }
    if (s == GI_OK)
        s = launch_interpolate_batched(reinterpret_cast<const InterpArgs *>(d + L.interp),
                                       reinterpret_cast<const uint32_t *>(d + L.pre[kPassInterp]), n,
                                       blocks[kPassInterp], st);
    return s;
}

} // namespace gi

using namespace gi;

extern "C" {

gi_status gi_batch_create(uint32_t n_views, uint32_t rays_per_probe, const gi_batch_tuning *tuning, gi_batch_t *out) {
    if (!out || n_views == 0 || n_views > GI_BATCH_MAX_VIEWS || rays_per_probe == 0 || rays_per_probe % 64 != 0) {
        set_error("gi_batch_create: bad view count, rays_per_probe or NULL output");
        return GI_ERR_INVALID_ARG;
    }
    *out = nullptr;
    gi_batch_tuning t = {2048u, 4u, 64u};
    if (tuning) t = *tuning;
    if (!tuning_ok(&t)) {
        set_error("gi_batch_create: tuning out of range");
        return GI_ERR_INVALID_ARG;
    }
    gi_batch_s *b = new gi_batch_s();
    b->n = n_views;
    b->nrcs.assign(n_views, nullptr);
    b->rpp = rays_per_probe;
    b->tuning = t;
    b->L = desc_layout(n_views);
    int dev = 0;
    gi_status s = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
    if (s == GI_OK) s = cuda_status(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev), "sm count");
    if (s == GI_OK) s = cuda_status(cudaMalloc(&b->d_desc, b->L.total), "cudaMalloc batch descriptors");
    for (int k = 0; k < 2 && s == GI_OK; ++k) {
        s = cuda_status(cudaMallocHost(&b->h_desc[k], b->L.total), "cudaMallocHost batch descriptors");
        if (s == GI_OK) memset(b->h_desc[k], 0, b->L.total);
        if (s == GI_OK) s = cuda_status(cudaEventCreateWithFlags(&b->used[k], cudaEventDisableTiming), "event");
    }
    if (s == GI_OK) s = cuda_status(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking), "capture stream");
    for (int k = 0; k < 4 && s == GI_OK; ++k) {
        s = cuda_status(cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking), "surrogate stream");
        if (s == GI_OK) s = cuda_status(cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming), "event");
    }
    if (s == GI_OK) s = cuda_status(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "event");
    if (s == GI_OK) s = ensure_moments();
    if (s != GI_OK) {
        free_batch(b);
        return s;
    }
    *out = b;
    return GI_OK;
}

gi_status gi_batch_set_tuning(gi_batch_t b, const gi_batch_tuning *tuning) {
    if (!b || !tuning_ok(tuning)) {
        set_error("gi_batch_set_tuning: NULL batch or tuning out of range");
        return GI_ERR_INVALID_ARG;
    }
    b->tuning = *tuning;
    gi_status s = cuda_status(cudaDeviceSynchronize(), "gi_batch_set_tuning sync");
    drop_graphs(b);
    return s;
}

gi_status gi_batch_set_surrogate(gi_batch_t b, gi_nrc_t nrc) {
    if (!b) {
        set_error("gi_batch_set_surrogate: NULL batch");
        return GI_ERR_INVALID_ARG;
    }
    b->nrcs.assign(b->n, nrc);
    b->surr = nrc != nullptr;
    return GI_OK;
}

gi_status gi_batch_set_view_surrogates(gi_batch_t b, const gi_nrc_t *nrcs) {
    if (!b) {
        set_error("gi_batch_set_view_surrogates: NULL batch");
        return GI_ERR_INVALID_ARG;
    }
    b->surr = false;
    for (uint32_t v = 0; v < b->n; ++v) {
        b->nrcs[v] = nrcs ? nrcs[v] : nullptr;
        b->surr = b->surr || b->nrcs[v] != nullptr;
    }
    return GI_OK;
}

gi_status gi_batch_destroy(gi_batch_t b) {
    if (!b) return GI_OK;
    cudaError_t e = cudaDeviceSynchronize();
    free_batch(b);
    return cuda_status(e, "gi_batch_destroy");
}

gi_status gi_batch_frame(gi_batch_t b, const gi_batch_view *views, uint32_t use_graph, gi_stream_t stream) {
    if (!b || !views) {
        set_error("gi_batch_frame: NULL batch or views");
        return GI_ERR_INVALID_ARG;
    }
    const uint32_t n = b->n;
    if (!views[0].cache) {
        set_error("gi_batch_frame: a view has no cache");
        return GI_ERR_INVALID_ARG;
    }
    const int key_dir = cache_key_dir(views[0].cache);
    for (uint32_t v = 0; v < n; ++v) {
        gi_status s = check_view(views[v], b->rpp, key_dir);
        if (s != GI_OK) return s;
        const gi_nrc_t routes = cache_route_nrc(views[v].cache);
        if (routes && routes != b->nrcs[v]) {
            set_error("gi_batch_frame: view %u routes far hits to a surrogate other than its own in the batch", v);
            return GI_ERR_INVALID_ARG;
        }
        if (cache_last_resolved(views[v].cache) > (int64_t)views[v].resolve_frame) {
            set_error("gi_batch_frame: view %u resolve frame %u precedes its cache's last resolved frame", v,
                      views[v].resolve_frame);
            return GI_ERR_INVALID_ARG;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int set = b->set;
    if (b->used_recorded[set]) {
        gi_status s = cuda_status(cudaEventSynchronize(b->used[set]), "batch descriptor reuse");
        if (s != GI_OK) return s;
    }
    // compaction checks first: they may move a table, and the descriptors below must see it
    for (uint32_t v = 0; v < n; ++v) {
        gi_status s = cache_before_update(views[v].cache, st);
        if (s != GI_OK) return s;
    }
    // block counts per pass and view
    const DescLayout &L = b->L;
    unsigned char *h = b->h_desc[set];
    uint32_t *pre[5];
    for (int k = 0; k < 5; ++k) {
        pre[k] = reinterpret_cast<uint32_t *>(h + L.pre[k]);
        pre[k][0] = 0;
    }
    unsigned long long total_records = 0;
    for (uint32_t v = 0; v < n; ++v) total_records += views[v].hits.n;
    const uint32_t res_total = (uint32_t)b->sms * b->tuning.resolve_blocks_per_sm;
    for (uint32_t v = 0; v < n; ++v) {
        const gi_batch_view &bv = views[v];
        const uint32_t tx = bv.probes.layout.tiles_x, ty = bv.probes.layout.tiles_y;
        const uint32_t cnt[5] = {
            ((tx + 15) / 16) * ((ty + 15) / 16),
            update_blocks_for(bv.hits.n, b->tuning.update_records_per_block),
            std::max<uint32_t>(1u, (uint32_t)((double)res_total * (double)bv.hits.n / (double)std::max(1ull, total_records))),
            b->nrcs[v] ? 0u
                       : (bv.probes.layout.num_probes * 4u + b->tuning.integrate_threads - 1u) /
                             b->tuning.integrate_threads,
            interp_grid_x(bv.view.width) * interp_grid_y(bv.view.height)};
        for (int k = 0; k < 5; ++k) pre[k][v + 1] = pre[k][v] + cnt[k];
        // far hits go to a surrogate only where the view's cache routes them to the view's surrogate
        reinterpret_cast<UpdateArgs *>(h + L.upd)[v] = cache_update_args(bv.cache, &bv.hits, &bv.view, bv.slot_ids);
        reinterpret_cast<ResolveArgs *>(h + L.res)[v] = cache_resolve_args(bv.cache, bv.resolve_frame);
        reinterpret_cast<SpawnArgs *>(h + L.spawn)[v] = spawn_args(&bv.gbuf, &bv.view, &bv.probes);
        reinterpret_cast<IntegrateArgs *>(h + L.integ)[v] = integrate_args(bv.cache, &bv.probes, bv.slot_ids, b->rpp, bv.env);
        reinterpret_cast<InterpArgs *>(h + L.interp)[v] = interp_args(&bv.gbuf, &bv.view, &bv.probes, bv.irradiance);
    }
    std::vector<uint32_t> blocks(5);
    for (int k = 0; k < 5; ++k) {
        blocks[k] = pre[k][n];
        pre[k][n + 1] = 0;  // the pass's work-item counter starts at zero every frame
    }
    gi_status s = GI_OK;
    if (use_graph && !b->surr) {
        if (!b->exec[set] || b->sig[set] != blocks) {
            if (b->exec[set]) cudaGraphExecDestroy(b->exec[set]);
            b->exec[set] = nullptr;
            cudaGraph_t g = nullptr;
            // capture on the batch's own stream (the caller's may be the legacy default stream)
            s = cuda_status(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal),
                            "cudaStreamBeginCapture");
            if (s == GI_OK) {
                gi_status se = enqueue_frame(b, set, blocks, key_dir, b->capture);
                gi_status sc = cuda_status(cudaStreamEndCapture(b->capture, &g), "cudaStreamEndCapture");
                s = se != GI_OK ? se : sc;
            }
            if (s == GI_OK) s = cuda_status(cudaGraphInstantiate(&b->exec[set], g, 0), "cudaGraphInstantiate");
            if (g) cudaGraphDestroy(g);
            if (s != GI_OK) return s;
            b->sig[set] = blocks;
        }
        s = cuda_status(cudaGraphLaunch(b->exec[set], st), "cudaGraphLaunch");
    } else {
        s = enqueue_frame(b, set, blocks, key_dir, st, views);
    }
    if (s != GI_OK) return s;
    s = cuda_status(cudaEventRecord(b->used[set], st), "batch event");
    if (s != GI_OK) return s;
    b->used_recorded[set] = true;
    b->set ^= 1;
    b->frames++;
    for (uint32_t v = 0; v < n; ++v) {
        cache_after_update(views[v].cache);
        cache_after_resolve(views[v].cache, views[v].resolve_frame);
    }
    return GI_OK;
}

} // extern "C"
