// Executor: one transform = permute in -> direct rectangles -> NUFFT sub-problems ->
// permute out, all enqueued on the plan's stream (Fig. 6 flow: inputs to chunk order,
// sub-transforms, row sums, outputs back to the caller's order).
#include <cuda_runtime.h>

#include <map>

#include "hvox_internal.h"

namespace hvox {

namespace {

size_t real_bytes(const Plan &p) { return p.prec == 1 ? sizeof(float) : sizeof(double); }

const double *weight_ptr(const Plan &p) { return p.has_weight ? p.weight.as<double>() : nullptr; }

cudaEvent_t take_event(Plan &p) {
    if (!p.event_pool.empty()) {
        cudaEvent_t e = p.event_pool.back();
        p.event_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    check_cuda(cudaEventCreate(&e), "cudaEventCreate");
    return e;
}

// Counts launches per stage and, when profiling, brackets each stage with events on the
// stream that runs it (the plan's stream or a NUFFT lane). Stage times are sums of the
// stages' durations, so stages that overlap on different lanes add up.
struct Profiler final : StageHook {
    Plan &p;
    std::map<cudaStream_t, cudaEvent_t> open;
    explicit Profiler(Plan &plan) : p(plan) {}
    void begin(int, cudaStream_t s) override {
        if (!p.profiling) return;
        cudaEvent_t e = take_event(p);
        check_cuda(cudaEventRecord(e, s), "cudaEventRecord");
        open[s] = e;
    }
    void end(int stage, int launches, cudaStream_t s) override {
        p.stage_launches[stage] += launches;
        if (!p.profiling) return;
        auto it = open.find(s);
        if (it == open.end()) return;
        cudaEvent_t b = take_event(p);
        check_cuda(cudaEventRecord(b, s), "cudaEventRecord");
        p.pending.push_back({stage, it->second, b});
        open.erase(it);
    }
};

template <typename T> NufftArgs<T> nufft_args(const Plan &p) {
    NufftArgs<T> a;
    a.w = p.es.w;
    a.beta = p.es.beta;
    a.isign = p.isign;
    a.ipsi = p.inv_psi.as<T>();
    a.pix_hi = p.pix_hi.as<float4>();
    a.pix_lo = p.pix_lo.as<float4>();
    a.vis_hi = p.vis_hi.as<float4>();
    a.vis_lo = p.vis_lo.as<float4>();
    a.pix_soa = p.pix_xyz.as<double>();
    a.vis_soa = p.vis_xyz.as<double>();
    a.n_pix = p.n_pix;
    a.n_vis = p.n_vis;
    a.cheb = p.cheb.as<T>();
    a.deg = p.cheb_deg;
    a.inv_tmax2 = p.cheb_inv_tmax2;
    return a;
}

// Lanes start after everything enqueued so far on the plan's stream.
void fork_lanes(Plan &p) {
    if (p.lanes.empty()) return;
    check_cuda(cudaEventRecord(p.fork_event, p.stream), "cudaEventRecord");
    for (auto &l : p.lanes) check_cuda(cudaStreamWaitEvent(l->stream, p.fork_event, 0), "cudaStreamWaitEvent");
}

// The plan's stream continues after every lane's work.
void join_lanes(Plan &p) {
    for (auto &l : p.lanes) {
        check_cuda(cudaEventRecord(l->done, l->stream), "cudaEventRecord");
        check_cuda(cudaStreamWaitEvent(p.stream, l->done, 0), "cudaStreamWaitEvent");
    }
}

template <typename T> void set_lane(NufftArgs<T> &a, const Plan &p, size_t b) {
    const Lane &l = *p.lanes[p.block_lane[b]];
    a.G1 = l.g1.as<typename CplxOf<T>::type>();
    a.G2 = l.g2.as<typename CplxOf<T>::type>();
    a.fft = p.block_fft[b];
}

}  // namespace

void collect_stats(Plan &p) {
    if (p.pending.empty()) return;
    check_cuda(cudaStreamSynchronize(p.stream), "collect_stats");
    for (auto &q : p.pending) {
        float ms = 0.f;
        check_cuda(cudaEventElapsedTime(&ms, q.a, q.b), "cudaEventElapsedTime");
        p.stage_ms[q.stage] += ms;
        p.event_pool.push_back(q.a);
        p.event_pool.push_back(q.b);
    }
    p.pending.clear();
}

void run_synthesize(Plan &p, const void *I, void *V) {
    cudaStream_t s = p.stream;
    const size_t re = real_bytes(p);
    Profiler prof(p);
    for (int t = 0; t < p.ntrans; ++t) {
        const char *It = (const char *)I + (size_t)t * p.n_pix * re;
        char *Vt = (char *)V + (size_t)t * p.n_vis * 2 * re;
        prof.begin(HVOX_STAGE_PERMUTE, s);
        launch_s2v_in(p.prec, It, p.pix_perm.as<int32_t>(), weight_ptr(p), p.n_pix, p.src.ptr, s);
        prof.end(HVOX_STAGE_PERMUTE, 1, s);
        prof.begin(HVOX_STAGE_ZERO, s);
        check_cuda(cudaMemsetAsync(p.acc.ptr, 0, (size_t)p.n_vis * 2 * re, s), "memset acc");
        prof.end(HVOX_STAGE_ZERO, 1, s);
        fork_lanes(p);
        if (p.n_items_s2v > 0) {
            prof.begin(HVOX_STAGE_DIRECT, s);
            const WorkItem *it = p.items_s2v.as<WorkItem>();
            if (p.plain)
                launch_direct_s2v_f64(it, p.n_items_s2v, p.vis_xyz.as<double>(), p.n_vis, p.pix_xyz.as<double>(),
                                      p.n_pix, p.src.as<double>(), p.acc.as<double2>(), p.isign, p.direct_vpt, s);
            else if (p.prec == 1)
                launch_direct_s2v_f32(it, p.n_items_s2v, p.vis_hi.as<float4>(), p.vis_lo.as<float4>(),
                                      p.pix_hi.as<float4>(), p.pix_lo.as<float4>(), p.src.as<float>(),
                                      p.acc.as<float2>(), p.isign, p.direct_vpt, s);
            else
                launch_direct_s2v_df(it, p.n_items_s2v, p.vis_hi.as<float4>(), p.vis_lo.as<float4>(),
                                     p.pix_hi.as<float4>(), p.pix_lo.as<float4>(), p.src.as<double>(),
                                     p.acc.as<double2>(), p.cis_tab.as<float4>(), p.isign, p.direct_vpt, s);
            prof.end(HVOX_STAGE_DIRECT, 1, s);
        }
        if (!p.dblocks.empty()) {
            if (p.prec == 1) {
                NufftArgs<float> a = nufft_args<float>(p);
                for (size_t b = 0; b < p.dblocks.size(); ++b) {
                    set_lane(a, p, b);
                    nufft_block_s2v<float>(p.dblocks[b], a, p.src.as<float>(), p.acc.as<float2>(), p.lanes[p.block_lane[b]]->stream, prof);
                }
            } else {
                NufftArgs<double> a = nufft_args<double>(p);
                for (size_t b = 0; b < p.dblocks.size(); ++b) {
                    set_lane(a, p, b);
                    nufft_block_s2v<double>(p.dblocks[b], a, p.src.as<double>(), p.acc.as<double2>(), p.lanes[p.block_lane[b]]->stream, prof);
                }
            }
        }
        join_lanes(p);
        prof.begin(HVOX_STAGE_PERMUTE, s);
        launch_s2v_out(p.prec, p.acc.ptr, p.vis_perm.as<int32_t>(), p.n_vis, Vt, s);
        prof.end(HVOX_STAGE_PERMUTE, 1, s);
        p.transforms++;
    }
}

void run_analyze(Plan &p, const void *V, void *I) {
    cudaStream_t s = p.stream;
    const size_t re = real_bytes(p);
    Profiler prof(p);
    for (int t = 0; t < p.ntrans; ++t) {
        const char *Vt = (const char *)V + (size_t)t * p.n_vis * 2 * re;
        char *It = (char *)I + (size_t)t * p.n_pix * re;
        prof.begin(HVOX_STAGE_PERMUTE, s);
        launch_v2s_in(p.prec, Vt, p.vis_perm.as<int32_t>(), p.n_vis, p.src.ptr, s);
        prof.end(HVOX_STAGE_PERMUTE, 1, s);
        prof.begin(HVOX_STAGE_ZERO, s);
        check_cuda(cudaMemsetAsync(p.acc.ptr, 0, (size_t)p.n_pix * re, s), "memset acc");
        prof.end(HVOX_STAGE_ZERO, 1, s);
        fork_lanes(p);
        if (p.n_items_v2s > 0) {
            prof.begin(HVOX_STAGE_DIRECT, s);
            const WorkItem *it = p.items_v2s.as<WorkItem>();
            if (p.plain)
                launch_direct_v2s_f64(it, p.n_items_v2s, p.pix_xyz.as<double>(), p.n_pix, p.vis_xyz.as<double>(),
                                      p.n_vis, p.src.as<double2>(), p.acc.as<double>(), p.isign, p.direct_vpt, s);
            else if (p.prec == 1)
                launch_direct_v2s_f32(it, p.n_items_v2s, p.pix_hi.as<float4>(), p.pix_lo.as<float4>(),
                                      p.vis_hi.as<float4>(), p.vis_lo.as<float4>(), p.src.as<float2>(),
                                      p.acc.as<float>(), p.isign, p.direct_vpt, s);
            else
                launch_direct_v2s_df(it, p.n_items_v2s, p.pix_hi.as<float4>(), p.pix_lo.as<float4>(),
                                     p.vis_hi.as<float4>(), p.vis_lo.as<float4>(), p.src.as<double2>(),
                                     p.acc.as<double>(), p.cis_tab.as<float4>(), p.isign, p.direct_vpt, s);
            prof.end(HVOX_STAGE_DIRECT, 1, s);
        }
        if (!p.dblocks.empty()) {
            if (p.prec == 1) {
                NufftArgs<float> a = nufft_args<float>(p);
                for (size_t b = 0; b < p.dblocks.size(); ++b) {
                    set_lane(a, p, b);
                    nufft_block_v2s<float>(p.dblocks[b], a, p.src.as<float2>(), p.acc.as<float>(), p.lanes[p.block_lane[b]]->stream, prof);
                }
            } else {
                NufftArgs<double> a = nufft_args<double>(p);
                for (size_t b = 0; b < p.dblocks.size(); ++b) {
                    set_lane(a, p, b);
                    nufft_block_v2s<double>(p.dblocks[b], a, p.src.as<double2>(), p.acc.as<double>(), p.lanes[p.block_lane[b]]->stream, prof);
                }
            }
        }
        join_lanes(p);
        prof.begin(HVOX_STAGE_PERMUTE, s);
        launch_v2s_out(p.prec, p.acc.ptr, p.pix_perm.as<int32_t>(), weight_ptr(p), p.n_pix, It, s);
        prof.end(HVOX_STAGE_PERMUTE, 1, s);
        p.transforms++;
    }
}

}  // namespace hvox
