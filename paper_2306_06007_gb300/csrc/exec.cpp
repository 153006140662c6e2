// Executor: one transform = permute in -> direct rectangles -> waves of NUFFT sub-problems
// -> permute out, all enqueued on the plan's stream (Fig. 6 flow: inputs to chunk order,
// sub-transforms, row sums, outputs back to the caller's order). The sub-problems of a
// wave share one launch per stage and one batched cuFFT set per grid shape (the parallel
// sub-transforms of Sect. 3); waves on different lanes run concurrently.
//
// The part between the permutations touches plan-owned buffers only, so after one eager
// call it is captured once per direction into a CUDA graph (the lanes forked from and
// joined into the capture stream) and replayed on the plan's stream; the permutations,
// whose pointers are the caller's, stay ordinary launches around the replay.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>

#include "hvox_internal.h"

namespace hvox {

namespace {

size_t real_bytes(const Plan &p) { return p.prec == 1 ? sizeof(float) : sizeof(double); }

const double *weight_ptr(const Plan &p) { return p.has_weight ? p.weight.as<double>() : nullptr; }

// Permutations of the caller's data (null: the caller works in chunk order).
const int32_t *pix_perm(const Plan &p) { return p.chunk_order ? nullptr : p.pix_perm.as<int32_t>(); }
const int32_t *vis_perm(const Plan &p) { return p.chunk_order ? nullptr : p.vis_perm.as<int32_t>(); }

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
// stages' durations, so stages that overlap on different lanes add up, and a bracket on a
// lane also counts the time its kernels wait for SMs held by concurrent work. The serial
// profiling mode runs every stage alone on the plan's stream, so there each bracket is
// the device time of its own launches.
// While a graph is captured (g set), launch counts and stage brackets go to the graph, and
// the brackets become event-record nodes whose events the graph owns.
struct Profiler final : StageHook {
    Plan &p;
    GraphRun *g = nullptr;
    std::map<cudaStream_t, cudaEvent_t> open;
    explicit Profiler(Plan &plan, GraphRun *graph = nullptr) : p(plan), g(graph) {}
    cudaEvent_t mark(cudaStream_t s) {
        cudaEvent_t e;
        if (g) {
            check_cuda(cudaEventCreate(&e), "cudaEventCreate");
            g->owned.push_back(e);
            check_cuda(cudaEventRecordWithFlags(e, s, cudaEventRecordExternal), "cudaEventRecordWithFlags");
        } else {
            e = take_event(p);
            check_cuda(cudaEventRecord(e, s), "cudaEventRecord");
        }
        return e;
    }
    void begin(int, cudaStream_t s) override {
        if (!p.profiling) return;
        open[s] = mark(s);
    }
    void end(int stage, int launches, cudaStream_t s) override {
        (g ? g->launches : p.stage_launches)[stage] += launches;
        if (!p.profiling) return;
        auto it = open.find(s);
        if (it == open.end()) return;
        cudaEvent_t b = mark(s);
        if (g)
            g->brackets.push_back({stage, it->second, b});
        else
            p.pending.push_back({stage, it->second, b});
        open.erase(it);
    }
};

template <typename T> NufftArgs<T> nufft_args(const Plan &p) {
    NufftArgs<T> a;
    a.w = p.es.w;
    a.beta = p.es.beta;
    a.isign = p.isign;
    a.descs = p.ddescs.as<NufftDev>();
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
    a.ppc_pix = p.ppc_pix;
    a.ppc_vis = p.ppc_vis;
    a.df_grids = p.df_grids;
    a.int_tile = p.int_tile;
    return a;
}

// Lanes start after everything enqueued so far on stream s. In the serialised profiling
// mode there is no fork: every sub-problem runs on s after the direct sums.
void fork_lanes(Plan &p, cudaStream_t s) {
    if (p.lanes.empty() || p.serial) return;
    check_cuda(cudaEventRecord(p.fork_event, s), "cudaEventRecord");
    for (auto &l : p.lanes) check_cuda(cudaStreamWaitEvent(l->stream, p.fork_event, 0), "cudaStreamWaitEvent");
}

// Stream s continues after every lane's work.
void join_lanes(Plan &p, cudaStream_t s) {
    if (p.serial) return;
    for (auto &l : p.lanes) {
        check_cuda(cudaEventRecord(l->done, l->stream), "cudaEventRecord");
        check_cuda(cudaStreamWaitEvent(s, l->done, 0), "cudaStreamWaitEvent");
    }
}

// Stream of a wave: its lane's, or s itself when profiling serially (the lane's grids and
// cuFFT plans are still used, one wave after another).
cudaStream_t wave_stream(const Plan &p, const Wave &w, cudaStream_t s) {
    return p.serial ? s : p.lanes[w.lane]->stream;
}

// Every wave of NUFFT sub-problems of one direction, each on its lane.
template <typename T, typename In, typename Out>
void run_waves(Plan &p, int dir, const In *src, Out *acc, cudaStream_t s, Profiler &prof) {
    const NufftArgs<T> a = nufft_args<T>(p);
    for (const Wave &w : p.waves) {
        Lane &l = *p.lanes[w.lane];
        if (dir == 0)
            nufft_wave_s2v<T>(w, a, l.g1.ptr, l.g2.ptr, reinterpret_cast<const T *>(src),
                              reinterpret_cast<typename CplxOf<T>::type *>(acc), wave_stream(p, w, s), prof);
        else
            nufft_wave_v2s<T>(w, a, l.g1.ptr, l.g2.ptr, reinterpret_cast<const typename CplxOf<T>::type *>(src),
                              reinterpret_cast<T *>(acc), wave_stream(p, w, s), prof);
    }
}

// sky -> vis between the permutations: src (chunk-ordered c_n) -> acc (chunk-ordered V).
void body_s2v(Plan &p, cudaStream_t s, Profiler &prof) {
    const size_t re = real_bytes(p);
    prof.begin(HVOX_STAGE_ZERO, s);
    check_cuda(cudaMemsetAsync(p.acc.ptr, 0, (size_t)p.n_vis * 2 * re, s), "memset acc");
    prof.end(HVOX_STAGE_ZERO, 1, s);
    fork_lanes(p, s);
    if (p.n_items_s2v > 0) {
        prof.begin(HVOX_STAGE_DIRECT, s);
        const WorkItem *it = p.items_s2v.as<WorkItem>();
        int *counter = p.item_counter.as<int>();
        check_cuda(cudaMemsetAsync(counter, 0, sizeof(int), s), "memset item counter");
        if (p.direct_f64)
            launch_direct_s2v_f64(it, p.n_items_s2v, counter, p.vis_xyz.as<double>(), p.n_vis, p.pix_xyz.as<double>(),
                                  p.n_pix, p.src.as<double>(), p.acc.as<double2>(), p.isign, p.direct_vpt, s);
        else if (p.prec == 1)
            launch_direct_s2v_f32(it, p.n_items_s2v, counter, p.vis_hi.as<float4>(), p.vis_lo.as<float4>(),
                                  p.pix_hi.as<float4>(), p.pix_lo.as<float4>(), p.src.as<float>(),
                                  p.acc.as<float2>(), p.isign, p.direct_vpt, s);
        else
            launch_direct_s2v_df(it, p.n_items_s2v, counter, p.vis_hi.as<float4>(), p.vis_lo.as<float4>(),
                                 p.pix_hi.as<float4>(), p.pix_lo.as<float4>(), p.src.as<double>(),
                                 p.acc.as<double2>(), p.cis_tab.as<float4>(), p.isign, p.direct_vpt, s);
        prof.end(HVOX_STAGE_DIRECT, 1, s);
    }
    if (!p.waves.empty()) {
        if (p.prec == 1)
            run_waves<float>(p, 0, p.src.as<float>(), p.acc.as<float2>(), s, prof);
        else
            run_waves<double>(p, 0, p.src.as<double>(), p.acc.as<double2>(), s, prof);
    }
    join_lanes(p, s);
}

// vis -> sky between the permutations: src (chunk-ordered V) -> acc (chunk-ordered I).
void body_v2s(Plan &p, cudaStream_t s, Profiler &prof) {
    const size_t re = real_bytes(p);
    prof.begin(HVOX_STAGE_ZERO, s);
    check_cuda(cudaMemsetAsync(p.acc.ptr, 0, (size_t)p.n_pix * re, s), "memset acc");
    prof.end(HVOX_STAGE_ZERO, 1, s);
    fork_lanes(p, s);
    if (p.n_items_v2s > 0) {
        prof.begin(HVOX_STAGE_DIRECT, s);
        const WorkItem *it = p.items_v2s.as<WorkItem>();
        int *counter = p.item_counter.as<int>() + 1;
        check_cuda(cudaMemsetAsync(counter, 0, sizeof(int), s), "memset item counter");
        if (p.direct_f64)
            launch_direct_v2s_f64(it, p.n_items_v2s, counter, p.pix_xyz.as<double>(), p.n_pix, p.vis_xyz.as<double>(),
                                  p.n_vis, p.src.as<double2>(), p.acc.as<double>(), p.isign, p.direct_vpt, s);
        else if (p.prec == 1)
            launch_direct_v2s_f32(it, p.n_items_v2s, counter, p.pix_hi.as<float4>(), p.pix_lo.as<float4>(),
                                  p.vis_hi.as<float4>(), p.vis_lo.as<float4>(), p.src.as<float2>(),
                                  p.acc.as<float>(), p.isign, p.direct_vpt, s);
        else
            launch_direct_v2s_df(it, p.n_items_v2s, counter, p.pix_hi.as<float4>(), p.pix_lo.as<float4>(),
                                 p.vis_hi.as<float4>(), p.vis_lo.as<float4>(), p.src.as<double2>(),
                                 p.acc.as<double>(), p.cis_tab.as<float4>(), p.isign, p.direct_vpt, s);
        prof.end(HVOX_STAGE_DIRECT, 1, s);
    }
    if (!p.waves.empty()) {
        if (p.prec == 1)
            run_waves<float>(p, 1, p.src.as<float2>(), p.acc.as<float>(), s, prof);
        else
            run_waves<double>(p, 1, p.src.as<double2>(), p.acc.as<double>(), s, prof);
    }
    join_lanes(p, s);
}

void body(Plan &p, int dir, cudaStream_t s, Profiler &prof) {
    if (dir == 0)
        body_s2v(p, s, prof);
    else
        body_v2s(p, s, prof);
}

bool graphs_wanted(const Plan &p) {
    if (p.plain || p.serial || p.graph_state < 0 || p.graphs_opt < 0) return false;
    return p.graphs_opt > 0 || !p.waves.empty();
}

// Gives up on graphs for this plan after a failed capture: ends the capture, drops the
// partial graph and the sticky capture error; later calls launch eagerly.
void abandon_capture(Plan &p) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(p.cap, &g);
    if (g) cudaGraphDestroy(g);
    (void)cudaGetLastError();
    p.graph_state = -1;
}

std::unique_ptr<GraphRun> capture(Plan &p, int dir) {
    auto g = std::make_unique<GraphRun>();
    if (!p.cap) check_cuda(cudaStreamCreateWithFlags(&p.cap, cudaStreamNonBlocking), "cudaStreamCreate");
    check_cuda(cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming), "cudaEventCreate");
    check_cuda(cudaStreamBeginCapture(p.cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    if (fault_hit("capture")) {
        abandon_capture(p);
        return nullptr;
    }
    try {
        Profiler prof(p, g.get());
        body(p, dir, p.cap, prof);
    } catch (const Error &) {
        abandon_capture(p);
        return nullptr;
    }
    cudaGraph_t graph = nullptr;
    if (cudaStreamEndCapture(p.cap, &graph) != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        (void)cudaGetLastError();
        p.graph_state = -1;
        return nullptr;
    }
    const cudaError_t e = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        p.graph_state = -1;
        return nullptr;
    }
    p.graph_state = 1;
    return g;
}

// Adds the stage times of a profiled replay to the plan's statistics.
void harvest(Plan &p, GraphRun &g) {
    if (!g.outstanding) return;
    check_cuda(cudaEventSynchronize(g.done), "cudaEventSynchronize");
    for (auto &b : g.brackets) {
        float ms = 0.f;
        check_cuda(cudaEventElapsedTime(&ms, b.a, b.b), "cudaEventElapsedTime");
        p.stage_ms[b.stage] += ms;
    }
    g.outstanding = false;
}

void execute(Plan &p, int dir) {
    cudaStream_t s = p.stream;
    if (!graphs_wanted(p) || p.eager_calls[dir] < 1) {
        p.eager_calls[dir]++;
        Profiler prof(p);
        body(p, dir, s, prof);
        return;
    }
    std::unique_ptr<GraphRun> &slot = p.graph[dir][p.profiling ? 1 : 0];
    if (!slot) slot = capture(p, dir);
    if (!slot) {
        Profiler prof(p);
        body(p, dir, s, prof);
        return;
    }
    GraphRun &g = *slot;
    harvest(p, g);
    check_cuda(cudaGraphLaunch(g.exec, s), "cudaGraphLaunch");
    for (int i = 0; i < HVOX_NUM_STAGES; ++i) p.stage_launches[i] += g.launches[i];
    if (p.profiling) {
        check_cuda(cudaEventRecord(g.done, s), "cudaEventRecord");
        g.outstanding = true;
    }
}

}  // namespace

template <typename T> NufftArgs<T> plan_nufft_args(const Plan &p) { return nufft_args<T>(p); }
template NufftArgs<float> plan_nufft_args<float>(const Plan &);
template NufftArgs<double> plan_nufft_args<double>(const Plan &);

void collect_stats(Plan &p) {
    for (auto &d : p.graph)
        for (auto &g : d)
            if (g) harvest(p, *g);
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
        launch_s2v_in(p.prec, It, pix_perm(p), weight_ptr(p), p.n_pix, p.src.ptr, s);
        prof.end(HVOX_STAGE_PERMUTE, 1, s);
        execute(p, 0);
        prof.begin(HVOX_STAGE_PERMUTE, s);
        launch_s2v_out(p.prec, p.acc.ptr, vis_perm(p), p.n_vis, Vt, s);
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
        launch_v2s_in(p.prec, Vt, vis_perm(p), p.n_vis, p.src.ptr, s);
        prof.end(HVOX_STAGE_PERMUTE, 1, s);
        execute(p, 1);
        prof.begin(HVOX_STAGE_PERMUTE, s);
        launch_v2s_out(p.prec, p.acc.ptr, pix_perm(p), weight_ptr(p), p.n_pix, It, s);
        prof.end(HVOX_STAGE_PERMUTE, 1, s);
        p.transforms++;
    }
}

namespace {

// The direct sums of one plan alone (FP64 kernels, or any plan outside a merged launch).
void direct_alone(Plan &p, int dir, cudaStream_t s) {
    const int64_t n = dir == 0 ? p.n_items_s2v : p.n_items_v2s;
    if (n <= 0) return;
    const WorkItem *it = (dir == 0 ? p.items_s2v : p.items_v2s).as<WorkItem>();
    int *counter = p.item_counter.as<int>() + dir;
    check_cuda(cudaMemsetAsync(counter, 0, sizeof(int), s), "memset item counter");
    if (dir == 0) {
        if (p.direct_f64)
            launch_direct_s2v_f64(it, n, counter, p.vis_xyz.as<double>(), p.n_vis, p.pix_xyz.as<double>(), p.n_pix,
                                  p.src.as<double>(), p.acc.as<double2>(), p.isign, p.direct_vpt, s);
        else if (p.prec == 1)
            launch_direct_s2v_f32(it, n, counter, p.vis_hi.as<float4>(), p.vis_lo.as<float4>(), p.pix_hi.as<float4>(),
                                  p.pix_lo.as<float4>(), p.src.as<float>(), p.acc.as<float2>(), p.isign,
                                  p.direct_vpt, s);
        else
            launch_direct_s2v_df(it, n, counter, p.vis_hi.as<float4>(), p.vis_lo.as<float4>(), p.pix_hi.as<float4>(),
                                 p.pix_lo.as<float4>(), p.src.as<double>(), p.acc.as<double2>(),
                                 p.cis_tab.as<float4>(), p.isign, p.direct_vpt, s);
    } else {
        if (p.direct_f64)
            launch_direct_v2s_f64(it, n, counter, p.pix_xyz.as<double>(), p.n_pix, p.vis_xyz.as<double>(), p.n_vis,
                                  p.src.as<double2>(), p.acc.as<double>(), p.isign, p.direct_vpt, s);
        else if (p.prec == 1)
            launch_direct_v2s_f32(it, n, counter, p.pix_hi.as<float4>(), p.pix_lo.as<float4>(), p.vis_hi.as<float4>(),
                                  p.vis_lo.as<float4>(), p.src.as<float2>(), p.acc.as<float>(), p.isign,
                                  p.direct_vpt, s);
        else
            launch_direct_v2s_df(it, n, counter, p.pix_hi.as<float4>(), p.pix_lo.as<float4>(), p.vis_hi.as<float4>(),
                                 p.vis_lo.as<float4>(), p.src.as<double2>(), p.acc.as<double>(),
                                 p.cis_tab.as<float4>(), p.isign, p.direct_vpt, s);
    }
    p.stage_launches[HVOX_STAGE_DIRECT] += 1;
}

// The job of a plan in a merged direct launch.
DirectJob job_of_plan(const Plan &p, int dir) {
    if (dir == 0)
        return {p.vis_hi.as<float4>(), p.vis_lo.as<float4>(), p.pix_hi.as<float4>(), p.pix_lo.as<float4>(),
                p.src.ptr,             p.acc.ptr,             (float)p.isign};
    return {p.pix_hi.as<float4>(), p.pix_lo.as<float4>(), p.vis_hi.as<float4>(), p.vis_lo.as<float4>(),
            p.src.ptr,             p.acc.ptr,             (float)p.isign};
}

// One merged launch over the work items of the plans in `group` (same kernel form and
// owners per thread). Its lists live in one stream-ordered allocation freed after it.
void direct_merged(const std::vector<Plan *> &group, int dir, int kind, int vpt, cudaStream_t s) {
    std::vector<DirectJob> jobs;
    std::vector<std::pair<int64_t, int>> order;  // (pairs, index into flat) for the sort
    std::vector<WorkItem> flat;
    std::vector<int> flat_job;
    for (size_t j = 0; j < group.size(); ++j) {
        jobs.push_back(job_of_plan(*group[j], dir));
        for (const WorkItem &w : group[j]->host_items[dir]) {
            order.push_back({(int64_t)(w.o1 - w.o0) * (int64_t)(w.s1 - w.s0), (int)flat.size()});
            flat.push_back(w);
            flat_job.push_back((int)j);
        }
    }
    // largest first (the schedule's assumption); ties keep plan order
    std::stable_sort(order.begin(), order.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
    const int64_t n = (int64_t)flat.size();
    const size_t b_items = sizeof(WorkItem) * (size_t)n, b_job = sizeof(int) * (size_t)n;
    const size_t b_jobs = sizeof(DirectJob) * jobs.size();
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    std::vector<char> host(up(b_items) + up(b_job) + up(b_jobs), 0);
    WorkItem *hi = reinterpret_cast<WorkItem *>(host.data());
    int *hj = reinterpret_cast<int *>(host.data() + up(b_items));
    for (int64_t i = 0; i < n; ++i) {
        hi[i] = flat[order[i].second];
        hj[i] = flat_job[order[i].second];
    }
    std::memcpy(host.data() + up(b_items) + up(b_job), jobs.data(), b_jobs);
    void *dev = nullptr;
    const size_t total = host.size() + 256;
    if (fault_hit("alloc")) fail(HVOX_ENOMEM, "batch work list: injected allocation failure");
    check_cuda(cudaMallocAsync(&dev, total, s), "cudaMallocAsync (batch work list)");
    char *d = static_cast<char *>(dev);
    check_cuda(cudaMemcpyAsync(d, host.data(), host.size(), cudaMemcpyHostToDevice, s), "copy batch work list");
    int *counter = reinterpret_cast<int *>(d + host.size());
    check_cuda(cudaMemsetAsync(counter, 0, sizeof(int), s), "memset batch counter");
    launch_direct_batch(kind, dir, reinterpret_cast<const WorkItem *>(d), n, counter,
                        reinterpret_cast<const DirectJob *>(d + up(b_items) + up(b_job)),
                        reinterpret_cast<const int *>(d + up(b_items)), group[0]->cis_tab.as<float4>(), vpt, s);
    check_cuda(cudaFreeAsync(dev, s), "cudaFreeAsync (batch work list)");
    for (Plan *p : group) p->stage_launches[HVOX_STAGE_DIRECT] += 1;
}

}  // namespace

int run_batch(const std::vector<Plan *> &plans, const std::vector<const void *> &in, const std::vector<void *> &out,
              int dir, cudaStream_t s) {
    // order after each plan's own stream
    for (Plan *p : plans) {
        if (!p->batch_event)
            check_cuda(cudaEventCreateWithFlags(&p->batch_event, cudaEventDisableTiming), "cudaEventCreate");
        if (p->stream != s) {
            check_cuda(cudaEventRecord(p->batch_event, p->stream), "cudaEventRecord");
            check_cuda(cudaStreamWaitEvent(s, p->batch_event, 0), "cudaStreamWaitEvent");
        }
    }
    // inputs to chunk order, accumulators cleared, lanes forked
    for (size_t i = 0; i < plans.size(); ++i) {
        Plan &p = *plans[i];
        const size_t re = real_bytes(p);
        if (dir == 0) {
            launch_s2v_in(p.prec, in[i], pix_perm(p), weight_ptr(p), p.n_pix, p.src.ptr, s);
            check_cuda(cudaMemsetAsync(p.acc.ptr, 0, (size_t)p.n_vis * 2 * re, s), "memset acc");
        } else {
            launch_v2s_in(p.prec, in[i], vis_perm(p), p.n_vis, p.src.ptr, s);
            check_cuda(cudaMemsetAsync(p.acc.ptr, 0, (size_t)p.n_pix * re, s), "memset acc");
        }
        p.stage_launches[HVOX_STAGE_PERMUTE] += 1;
        p.stage_launches[HVOX_STAGE_ZERO] += 1;
        fork_lanes(p, s);
    }
    // direct sums: merged per (kernel form, owners per thread); FP64 kernels alone
    int launches = 0;
    std::map<std::pair<int, int>, std::vector<Plan *>> groups;
    for (Plan *p : plans) {
        if ((dir == 0 ? p->n_items_s2v : p->n_items_v2s) <= 0) continue;
        if (p->direct_f64) {
            direct_alone(*p, dir, s);
            ++launches;
        } else {
            groups[{p->prec == 1 ? 0 : 1, p->direct_vpt}].push_back(p);
        }
    }
    for (auto &g : groups) {
        if (g.second.size() == 1)
            direct_alone(*g.second[0], dir, s);
        else
            direct_merged(g.second, dir, g.first.first, g.first.second, s);
        ++launches;
    }
    // NUFFT sub-problems on each plan's lanes, outputs back to the callers' order
    for (size_t i = 0; i < plans.size(); ++i) {
        Plan &p = *plans[i];
        Profiler prof(p);
        if (!p.waves.empty()) {
            if (p.prec == 1) {
                if (dir == 0)
                    run_waves<float>(p, 0, p.src.as<float>(), p.acc.as<float2>(), s, prof);
                else
                    run_waves<float>(p, 1, p.src.as<float2>(), p.acc.as<float>(), s, prof);
            } else {
                if (dir == 0)
                    run_waves<double>(p, 0, p.src.as<double>(), p.acc.as<double2>(), s, prof);
                else
                    run_waves<double>(p, 1, p.src.as<double2>(), p.acc.as<double>(), s, prof);
            }
        }
        join_lanes(p, s);
        if (dir == 0)
            launch_s2v_out(p.prec, p.acc.ptr, vis_perm(p), p.n_vis, out[i], s);
        else
            launch_v2s_out(p.prec, p.acc.ptr, pix_perm(p), weight_ptr(p), p.n_pix, out[i], s);
        p.stage_launches[HVOX_STAGE_PERMUTE] += 1;
        p.transforms++;
    }
    // each plan's own stream continues after the call
    cudaEvent_t done = plans[0]->batch_event;
    check_cuda(cudaEventRecord(done, s), "cudaEventRecord");
    for (Plan *p : plans)
        if (p->stream != s) check_cuda(cudaStreamWaitEvent(p->stream, done, 0), "cudaStreamWaitEvent");
    return launches;
}

// A (x + j y) = A x + j A y: both real skies through the ordinary path, then V += j V'.
void run_synthesize_complex(Plan &p, const void *I, void *V) {
    const size_t re = real_bytes(p);
    if (p.cplx_sky.bytes < 2 * (size_t)p.n_pix * re) p.cplx_sky.alloc(2 * (size_t)p.n_pix * re);
    if (p.cplx_vis.bytes < 2 * (size_t)p.n_vis * re) p.cplx_vis.alloc(2 * (size_t)p.n_vis * re);
    char *x = (char *)p.cplx_sky.ptr, *y = x + (size_t)p.n_pix * re;
    launch_split_complex(p.prec, I, p.n_pix, x, y, p.stream);
    run_synthesize(p, x, V);
    run_synthesize(p, y, p.cplx_vis.ptr);
    launch_add_j(p.prec, V, p.cplx_vis.ptr, p.n_vis, p.stream);
}

// A^H v = Re(A^H v) + j Re(A^H (-j v)): the ordinary (real-part) adjoint twice.
void run_analyze_complex(Plan &p, const void *V, void *I) {
    const size_t re = real_bytes(p);
    if (p.cplx_sky.bytes < 2 * (size_t)p.n_pix * re) p.cplx_sky.alloc(2 * (size_t)p.n_pix * re);
    if (p.cplx_vis.bytes < 2 * (size_t)p.n_vis * re) p.cplx_vis.alloc(2 * (size_t)p.n_vis * re);
    char *x = (char *)p.cplx_sky.ptr, *y = x + (size_t)p.n_pix * re;
    run_analyze(p, V, x);
    launch_times_mj(p.prec, V, p.n_vis, p.cplx_vis.ptr, p.stream);
    run_analyze(p, p.cplx_vis.ptr, y);
    launch_join_complex(p.prec, x, y, p.n_pix, I, p.stream);
}

}  // namespace hvox
