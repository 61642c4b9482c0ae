// serve.cpp - continuous-batching request engine and its one-size-per-launch
// baseline.  Not a construct of the paper: a serving form of the same decoder
// (every request is decoded exactly as a solo call would decode it).
//
// polar_serve: requests arrive at given times.  A producer loop releases each
// request once it has arrived and the LLR arena (a fixed HBM budget) has room
// for it: the batch of requests released together is gathered into a pinned
// host mirror of the arena (same offsets), copied to the arena in one
// transfer (two when it wraps), and a published-count is advanced on the
// device behind it on the same stream; releases are at least kReleaseTick
// apart, so that arrivals in between share one batch.  One persistent kernel (scs_serve_kernel) keeps
// every warp busy: a warp that finishes a request claims the next index,
// waits (bounded) until it is published, and decodes it, so new requests
// start while older ones are still on the GPU.  Arena space is handed out in
// request order and returned when the oldest outstanding requests complete
// (completion flags in host-mapped memory).  Latency = completion time
// (device clock, aligned to the host clock at start) - arrival time.
//
// polar_serve_baseline: every `interval` seconds the requests that have
// arrived are grouped by (code, D, L) and each group is decoded by its own
// scs_decode_batch launch; a request completes when its group's launch does.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "plan.h"

namespace polarscs {
int serve_codes(const polar_plan_set *set, const void **out);
int launch_scs_serve(const polar_plan_set *set, const void *codes, const int4 *d_frames, int B, int Dmax,
                     const float *d_arena, const long long *d_llr_off, uint32_t *d_info, const long long *d_info_off,
                     float *d_pm, int8_t *d_status, const unsigned long long *d_head, const int *h_abort,
                     unsigned char *h_done, unsigned long long *d_t_done, unsigned long long *d_t_start, int *d_error,
                     unsigned long long wait_ns, unsigned *d_counter, uint32_t *d_scratch, size_t scratch_bytes,
                     int wpb_pref, cudaStream_t stream);
size_t serve_scratch_bytes(const polar_plan_set *set, int Dmax);
int read_device_ns(unsigned long long *d_out, cudaStream_t s);
int launch_scs_decode(const polar_plan *p, const DeviceTables *dt, const float *d_llr, int B, int D, int L,
                      uint32_t *d_info, float *d_pm, int8_t *d_status, uint32_t *d_stats, cudaStream_t stream);
}  // namespace polarscs

using namespace polarscs;
using Clock = std::chrono::steady_clock;

namespace {

double seconds_since(Clock::time_point t0) { return std::chrono::duration<double>(Clock::now() - t0).count(); }

// Shortest interval between two releases of polar_serve.  Each release costs
// two or three small host-to-device copies; released as fast as the loop
// turns, 1 M requests/s became ~10^5 releases/s, more copies than the copy
// engine retires, and requests waited 4-5 ms (p50) for their copy.  With
// 20 us between releases the p50 wait is 0.09 ms at 1 M requests/s and
// 0.08 ms at 0.2 M (GB300; 50 us: 0.10 ms, 100 us: 0.15 ms).
constexpr double kReleaseTick = 20e-6;

// RAII owners for the engine's device and pinned buffers
struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes < 16 ? 16 : bytes); }
};
struct HostBuf {
    void *p = nullptr;
    ~HostBuf() {
        if (p) cudaFreeHost(p);
    }
    cudaError_t alloc(size_t bytes, unsigned flags) { return cudaHostAlloc(&p, bytes < 16 ? 16 : bytes, flags); }
};

// request layout shared by both engines: sizes, arena placement (contiguous,
// skipping to the arena start when a frame would cross its end), virtual
// positions for the space test
struct Layout {
    std::vector<int> N, words;
    std::vector<long long> off, vstart;
    long long arena = 0;
};

int make_layout(const polar_plan_set *set, const int32_t *req, int R, long long arena, Layout *L, int *Dmax) {
    L->N.resize(size_t(R));
    L->words.resize(size_t(R));
    L->off.resize(size_t(R));
    L->vstart.resize(size_t(R));
    L->arena = arena;
    long long pos = 0, v = 0;
    *Dmax = 1;
    for (int r = 0; r < R; ++r) {
        const int pi = req[4 * size_t(r)];
        if (pi < 0 || pi >= int(set->plans.size())) return POLAR_EINVAL;
        const int D = req[4 * size_t(r) + 1], Lr = req[4 * size_t(r) + 2];
        if (D < 1 || D > POLAR_MAX_D_GPU || Lr < 1 || Lr > POLAR_MAX_L_GPU) return POLAR_EINVAL;
        *Dmax = std::max(*Dmax, D);
        const int N = set->plans[size_t(pi)]->N;
        if (N > arena) return POLAR_EINVAL;
        L->N[size_t(r)] = N;
        L->words[size_t(r)] = (set->plans[size_t(pi)]->Kmsg + 31) / 32;
        if (pos + N > arena) {  // skip the arena's tail
            v += arena - pos;
            pos = 0;
        }
        L->off[size_t(r)] = pos;
        L->vstart[size_t(r)] = v;
        pos += N;
        v += N;
    }
    return 0;
}

}  // namespace

extern "C" int polar_serve(const polar_plan_set *set, const int32_t *req, const double *arrival_s, int R,
                           const float *pool_llr, const int64_t *pool_off, int P, int64_t arena_floats,
                           double wait_s, float *pm_out, int8_t *status_out, uint32_t *info_out,
                           const int64_t *info_off, double *latency_out, double *service_out, double *report) {
    TraceRange trace("polar_serve");
    if (!set || !req || !arrival_s || R < 1 || !pool_llr || !pool_off || P < 1 || arena_floats < 1 || !pm_out ||
        !status_out || !latency_out || !report || wait_s <= 0.0)
        return POLAR_EINVAL;
    for (int r = 0; r < R; ++r) {
        const int p = req[4 * size_t(r) + 3];
        if (p < 0 || p >= P) return POLAR_EINVAL;
        if (r && arrival_s[r] < arrival_s[r - 1]) return POLAR_EINVAL;  // arrivals in order
    }
    Layout lay;
    int Dmax = 1;
    int rc = make_layout(set, req, R, arena_floats, &lay, &Dmax);
    if (rc) return rc;
    for (int p = 0; p < P; ++p)
        if (pool_off[p] < 0) return POLAR_EINVAL;

    const void *codes = nullptr;
    rc = serve_codes(set, &codes);
    if (rc) return rc;

    // device-side descriptors of every request (known up front; only their
    // arrival is dynamic)
    std::vector<int4> frames(static_cast<size_t>(R));
    std::vector<long long> ioff(static_cast<size_t>(R));
    long long wsum = 0;
    for (int r = 0; r < R; ++r) {
        frames[size_t(r)] = make_int4(req[4 * size_t(r)], req[4 * size_t(r) + 1], req[4 * size_t(r) + 2], 0);
        ioff[size_t(r)] = info_off ? (long long)info_off[r] : wsum;
        wsum += lay.words[size_t(r)];
    }
    long long out_words = wsum;
    if (info_off)
        for (int r = 0; r < R; ++r) out_words = std::max(out_words, ioff[size_t(r)] + lay.words[size_t(r)]);

    cudaError_t e = cudaSuccess;
    DevBuf d_arena, d_frames, d_loff, d_ioff, d_info, d_pm, d_st, d_tdone, d_tstart, d_head, d_err, d_cnt, d_scr, d_gt;
    HostBuf h_done, h_abort, h_head, h_tdone, h_tstart, h_mirror;
    const size_t scr_bytes = serve_scratch_bytes(set, Dmax);
    if ((e = d_arena.alloc(size_t(arena_floats) * 4)) != cudaSuccess || (e = d_frames.alloc(sizeof(int4) * R)) ||
        (e = d_loff.alloc(8 * size_t(R))) || (e = d_ioff.alloc(8 * size_t(R))) ||
        (e = d_info.alloc(4 * size_t(out_words))) || (e = d_pm.alloc(4 * size_t(R))) || (e = d_st.alloc(size_t(R))) ||
        (e = d_tdone.alloc(8 * size_t(R))) || (e = d_tstart.alloc(8 * size_t(R))) || (e = d_head.alloc(8)) ||
        (e = d_err.alloc(4)) || (e = d_cnt.alloc(4)) ||
        (e = d_scr.alloc(scr_bytes)) || (e = d_gt.alloc(8)) || (e = h_done.alloc(size_t(R), cudaHostAllocMapped)) ||
        (e = h_abort.alloc(4, cudaHostAllocMapped)) || (e = h_head.alloc(8 * 4096, 0)) ||
        (e = h_tdone.alloc(8 * size_t(R), 0)) || (e = h_tstart.alloc(8 * size_t(R), 0)) ||
        (e = h_mirror.alloc(size_t(arena_floats) * 4, 0)))
        return cuda_status(e);
    float *mirror = static_cast<float *>(h_mirror.p);
    volatile unsigned char *done = static_cast<volatile unsigned char *>(h_done.p);
    volatile int *abort_flag = static_cast<volatile int *>(h_abort.p);
    std::memset(h_done.p, 0, size_t(R));
    *abort_flag = 0;
    unsigned char *d_done = nullptr;
    int *d_abort = nullptr;
    if ((e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&d_done), h_done.p, 0)) ||
        (e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&d_abort), h_abort.p, 0)))
        return cuda_status(e);

    cudaStream_t ks = nullptr, cs = nullptr;
    if ((e = cudaStreamCreateWithFlags(&ks, cudaStreamNonBlocking)) ||
        (e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)))
        return cuda_status(e);
    auto cleanup = [&]() {
        cudaStreamDestroy(ks);
        cudaStreamDestroy(cs);
    };
    if ((e = cudaMemcpy(d_frames.p, frames.data(), sizeof(int4) * R, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(d_loff.p, lay.off.data(), 8 * size_t(R), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(d_ioff.p, ioff.data(), 8 * size_t(R), cudaMemcpyHostToDevice)) ||
        (e = cudaMemset(d_head.p, 0, 8)) || (e = cudaMemset(d_err.p, 0, 4)) || (e = cudaMemset(d_cnt.p, 0, 4)) ||
        (e = cudaMemset(d_st.p, 0x7f, size_t(R)))) {
        cleanup();
        return cuda_status(e);
    }

    // align the device clock to the host clock: the tightest of several
    // round trips (the first launch of a process can be slow)
    unsigned long long gt0 = 0;
    Clock::time_point h0{};
    double best_rtt = -1.0;
    for (int trial = 0; trial < 8; ++trial) {
        unsigned long long g = 0;
        const Clock::time_point ha = Clock::now();
        rc = read_device_ns(static_cast<unsigned long long *>(d_gt.p), ks);
        if (rc == 0) e = cudaStreamSynchronize(ks);
        const Clock::time_point hb = Clock::now();
        if (rc == 0 && e == cudaSuccess) e = cudaMemcpy(&g, d_gt.p, 8, cudaMemcpyDeviceToHost);
        if (rc || e != cudaSuccess) {
            cleanup();
            return rc ? rc : cuda_status(e);
        }
        const double rtt = std::chrono::duration<double>(hb - ha).count();
        if (best_rtt < 0.0 || rtt < best_rtt) {
            best_rtt = rtt;
            gt0 = g;
            h0 = ha + (hb - ha) / 2;
        }
    }

    rc = launch_scs_serve(set, codes, static_cast<const int4 *>(d_frames.p), R, Dmax,
                          static_cast<const float *>(d_arena.p), static_cast<const long long *>(d_loff.p),
                          static_cast<uint32_t *>(d_info.p), static_cast<const long long *>(d_ioff.p),
                          static_cast<float *>(d_pm.p), static_cast<int8_t *>(d_st.p),
                          static_cast<const unsigned long long *>(d_head.p), d_abort, d_done,
                          static_cast<unsigned long long *>(d_tdone.p), static_cast<unsigned long long *>(d_tstart.p),
                          static_cast<int *>(d_err.p),
                          (unsigned long long)(wait_s * 1e9), static_cast<unsigned *>(d_cnt.p),
                          static_cast<uint32_t *>(d_scr.p), scr_bytes, 0, ks);
    if (rc) {
        cleanup();
        return rc;
    }

    // producer: release requests in arrival order as the arena allows
    unsigned long long *head_stage = static_cast<unsigned long long *>(h_head.p);
    const Clock::time_point t_start = Clock::now();
    int published = 0, oldest = 0, slot = 0, max_inflight = 0;
    long long stalls = 0;
    bool aborted = false;
    const double last_arrival = arrival_s[R - 1];
    double last_release = -kReleaseTick;
    while (published < R) {
        const double now = seconds_since(t_start);
        if (now - last_release < kReleaseTick) {
            std::this_thread::sleep_for(std::chrono::microseconds(2));
            continue;
        }
        while (oldest < published && done[oldest]) ++oldest;
        const long long base = oldest < published ? lay.vstart[size_t(oldest)] : lay.vstart[size_t(published)];
        int r_end = published;
        while (r_end < R && arrival_s[r_end] <= now && lay.vstart[size_t(r_end)] + lay.N[size_t(r_end)] - base <= lay.arena)
            ++r_end;
        if (r_end == published) {
            if (arrival_s[published] <= now) ++stalls;  // arrived, but the arena is full
            if (now > last_arrival + wait_s) {
                aborted = true;
                break;
            }
            std::this_thread::sleep_for(std::chrono::microseconds(2));
            continue;
        }
        // gather the new requests' LLRs into the mirror (their arena
        // places are free: arena admission returned them only after the
        // requests that used them completed, copies included), then copy
        // each run contiguous in the arena (one, two when the batch wraps)
        for (int q = published; q < r_end; ++q)
            std::memcpy(mirror + lay.off[size_t(q)], pool_llr + pool_off[req[4 * size_t(q) + 3]],
                        size_t(lay.N[size_t(q)]) * 4);
        int r = published;
        while (r < r_end && e == cudaSuccess) {
            int q = r + 1;
            long long len = lay.N[size_t(r)];
            while (q < r_end && lay.off[size_t(q)] == lay.off[size_t(r)] + len) {
                len += lay.N[size_t(q)];
                ++q;
            }
            e = cudaMemcpyAsync(static_cast<float *>(d_arena.p) + lay.off[size_t(r)], mirror + lay.off[size_t(r)],
                                size_t(len) * 4, cudaMemcpyHostToDevice, cs);
            r = q;
        }
        head_stage[slot] = (unsigned long long)r_end;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_head.p, head_stage + slot, 8, cudaMemcpyHostToDevice, cs);
        if (e != cudaSuccess) {
            aborted = true;
            break;
        }
        if (++slot == 4096) {  // the staging ring is reused: let its copies drain
            slot = 0;
            cudaStreamSynchronize(cs);
        }
        published = r_end;
        last_release = now;
        max_inflight = std::max(max_inflight, published - oldest);
    }
    // wait (bounded) for the kernel to finish
    const Clock::time_point t_wait = Clock::now();
    while (!aborted && cudaStreamQuery(ks) == cudaErrorNotReady) {
        if (seconds_since(t_wait) > wait_s) {
            aborted = true;
            break;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    if (aborted) *abort_flag = 1;
    cudaError_t es = cudaStreamSynchronize(ks);
    cudaStreamSynchronize(cs);
    int err_host = 0;
    if (es == cudaSuccess) es = cudaMemcpy(&err_host, d_err.p, 4, cudaMemcpyDeviceToHost);
    if (es == cudaSuccess) es = cudaMemcpy(pm_out, d_pm.p, 4 * size_t(R), cudaMemcpyDeviceToHost);
    if (es == cudaSuccess) es = cudaMemcpy(status_out, d_st.p, size_t(R), cudaMemcpyDeviceToHost);
    if (es == cudaSuccess) es = cudaMemcpy(h_tdone.p, d_tdone.p, 8 * size_t(R), cudaMemcpyDeviceToHost);
    if (es == cudaSuccess) es = cudaMemcpy(h_tstart.p, d_tstart.p, 8 * size_t(R), cudaMemcpyDeviceToHost);
    if (es == cudaSuccess && info_out) es = cudaMemcpy(info_out, d_info.p, 4 * size_t(out_words), cudaMemcpyDeviceToHost);
    cleanup();
    if (es != cudaSuccess) return cuda_status(es);
    const unsigned long long *td = static_cast<const unsigned long long *>(h_tdone.p);
    const unsigned long long *ts = static_cast<const unsigned long long *>(h_tstart.p);
    const double start_off = std::chrono::duration<double>(t_start - h0).count();  // host start relative to gt0
    double last = 0.0;
    int completed = 0;
    for (int r = 0; r < R; ++r) {
        if (!done[r]) {
            latency_out[r] = std::nan("");
            if (service_out) service_out[r] = std::nan("");
            continue;
        }
        if (service_out) service_out[r] = double((long long)(td[r] - ts[r])) * 1e-9;  // on the device clock
        ++completed;
        const double t_done_s = double((long long)(td[r] - gt0)) * 1e-9 - start_off;  // since t_start
        latency_out[r] = t_done_s - arrival_s[r];
        last = std::max(last, t_done_s);
    }
    report[0] = last;                       // seconds from start to the last completion
    report[1] = double(stalls);             // producer polls that found the arena full
    report[2] = double(err_host || aborted);
    report[3] = double(max_inflight);       // most requests between oldest outstanding and newest published
    report[4] = double(completed);
    report[5] = double(arena_floats) * 4.0;  // HBM budget of the arena in bytes
    return (err_host || aborted || completed != R) ? POLAR_ETIMEOUT : 0;
}

namespace {
struct GroupDone {
    std::vector<int> reqs;
    Clock::time_point *done_at;
    const Clock::time_point *t0;
    std::vector<double> *done_s;
    int8_t *st_host;
    float *pm_host;
    float *pm_out;
    int8_t *st_out;
};

void CUDART_CB group_done_cb(void *arg) {
    GroupDone *g = static_cast<GroupDone *>(arg);
    const double t = std::chrono::duration<double>(Clock::now() - *g->t0).count();
    for (size_t i = 0; i < g->reqs.size(); ++i) {
        const int r = g->reqs[i];
        (*g->done_s)[size_t(r)] = t;
        g->pm_out[r] = g->pm_host[i];
        g->st_out[r] = g->st_host[i];
    }
}
}  // namespace

extern "C" int polar_serve_baseline(const polar_plan_set *set, const int32_t *req, const double *arrival_s, int R,
                                    const float *pool_llr, const int64_t *pool_off, int P, int64_t arena_floats,
                                    double interval_s, double wait_s, float *pm_out, int8_t *status_out,
                                    double *latency_out, double *report) {
    TraceRange trace("polar_serve_baseline");
    if (!set || !req || !arrival_s || R < 1 || !pool_llr || !pool_off || P < 1 || arena_floats < 1 || !pm_out ||
        !status_out || !latency_out || !report || interval_s <= 0.0 || wait_s <= 0.0)
        return POLAR_EINVAL;
    for (int r = 0; r < R; ++r) {
        const int p = req[4 * size_t(r) + 3];
        if (p < 0 || p >= P) return POLAR_EINVAL;
        if (r && arrival_s[r] < arrival_s[r - 1]) return POLAR_EINVAL;
    }
    Layout lay;
    int Dmax = 1;
    int rc = make_layout(set, req, R, arena_floats, &lay, &Dmax);
    if (rc) return rc;
    std::vector<const DeviceTables *> tabs(static_cast<size_t>(set->plans.size()));
    for (size_t i = 0; i < set->plans.size(); ++i) {
        rc = plan_device(set->plans[i], &tabs[i]);
        if (rc) return rc;
    }
    // staging: pinned host copy of the group's LLRs, device arena, outputs
    HostBuf h_stage, h_pm, h_st;
    DevBuf d_arena, d_info, d_pm, d_st;
    cudaError_t e;
    if ((e = h_stage.alloc(size_t(arena_floats) * 4, 0)) || (e = h_pm.alloc(4 * size_t(R), 0)) ||
        (e = h_st.alloc(size_t(R), 0)) || (e = d_arena.alloc(size_t(arena_floats) * 4)) ||
        (e = d_info.alloc(4 * size_t(arena_floats))) || (e = d_pm.alloc(4 * size_t(R))) || (e = d_st.alloc(size_t(R))))
        return cuda_status(e);
    cudaStream_t s = nullptr;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking))) return cuda_status(e);
    std::vector<double> done_s(static_cast<size_t>(R), -1.0);
    std::vector<std::unique_ptr<GroupDone>> groups;
    std::vector<cudaEvent_t> events;
    const Clock::time_point t0 = Clock::now();
    // the arena (and its pinned host mirror) is a ring of whole batches; a
    // batch waits only for the earlier batches whose region it overwrites
    // (checked against every batch in flight)
    long long ring_pos = 0;
    std::vector<std::tuple<long long, long long, cudaEvent_t>> inflight;  // [start, end), done event; oldest first
    size_t inflight_head = 0;
    int published = 0, batches = 0;
    long long stalls = 0;
    bool failed = false;
    double next_tick = interval_s;
    while (published < R && !failed) {
        double now = std::chrono::duration<double>(Clock::now() - t0).count();
        if (now < next_tick && arrival_s[published] > now) {
            std::this_thread::sleep_for(std::chrono::microseconds(5));
            continue;
        }
        next_tick = now + interval_s;
        int r_end = published;
        while (r_end < R && arrival_s[r_end] <= now) ++r_end;
        if (r_end == published) continue;
        // group by (code, D, L) in arrival order
        std::map<std::tuple<int, int, int>, std::vector<int>> by_cfg;
        for (int r = published; r < r_end; ++r)
            by_cfg[std::make_tuple(req[4 * size_t(r)], req[4 * size_t(r) + 1], req[4 * size_t(r) + 2])].push_back(r);
        for (auto &kv : by_cfg) {
            const int pi = std::get<0>(kv.first), D = std::get<1>(kv.first), Lr = std::get<2>(kv.first);
            const polar_plan *pl = set->plans[size_t(pi)];
            const std::vector<int> &rs = kv.second;
            // split the group into chunks that fit the arena
            size_t i0 = 0;
            while (i0 < rs.size() && !failed) {
                size_t i1 = i0;
                long long need = 0;
                while (i1 < rs.size() && need + pl->N <= arena_floats) {
                    need += pl->N;
                    ++i1;
                }
                if (ring_pos + need > arena_floats) ring_pos = 0;
                // after a wrap, regions are not in age order: check every batch
                // still in flight, then retire the completed ones at the front
                for (size_t q = inflight_head; q < inflight.size(); ++q) {
                    const auto &f = inflight[q];
                    if (std::get<0>(f) < ring_pos + need && ring_pos < std::get<1>(f) &&
                        cudaEventQuery(std::get<2>(f)) == cudaErrorNotReady) {
                        ++stalls;
                        cudaEventSynchronize(std::get<2>(f));
                    }
                }
                while (inflight_head < inflight.size() && cudaEventQuery(std::get<2>(inflight[inflight_head])) == cudaSuccess)
                    ++inflight_head;
                const int n = int(i1 - i0);
                float *stage = static_cast<float *>(h_stage.p) + ring_pos;
                for (int j = 0; j < n; ++j) {
                    const int r = rs[i0 + size_t(j)];
                    std::memcpy(stage + size_t(j) * pl->N, pool_llr + pool_off[req[4 * size_t(r) + 3]], size_t(pl->N) * 4);
                }
                float *dl = static_cast<float *>(d_arena.p) + ring_pos;
                e = cudaMemcpyAsync(dl, stage, size_t(need) * 4, cudaMemcpyHostToDevice, s);
                // outputs go to fixed device and host buffers: the stream orders
                // each batch's decode, read-back and completion callback
                int lrc = e == cudaSuccess ? launch_scs_decode(pl, tabs[size_t(pi)], dl, n, D, Lr,
                                                               static_cast<uint32_t *>(d_info.p),
                                                               static_cast<float *>(d_pm.p), static_cast<int8_t *>(d_st.p),
                                                               nullptr, s)
                                           : cuda_status(e);
                if (lrc) {
                    failed = true;
                    break;
                }
                auto g = std::make_unique<GroupDone>();
                g->reqs.assign(rs.begin() + long(i0), rs.begin() + long(i1));
                g->t0 = &t0;
                g->done_s = &done_s;
                g->pm_host = static_cast<float *>(h_pm.p);
                g->st_host = static_cast<int8_t *>(h_st.p);
                g->pm_out = pm_out;
                g->st_out = status_out;
                cudaMemcpyAsync(g->pm_host, d_pm.p, 4 * size_t(n), cudaMemcpyDeviceToHost, s);
                cudaMemcpyAsync(g->st_host, d_st.p, size_t(n), cudaMemcpyDeviceToHost, s);
                cudaLaunchHostFunc(s, group_done_cb, g.get());
                cudaEvent_t ev = nullptr;
                cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
                cudaEventRecord(ev, s);
                events.push_back(ev);
                inflight.emplace_back(ring_pos, ring_pos + need, ev);
                groups.push_back(std::move(g));
                ring_pos += need;
                ++batches;
                i0 = i1;
            }
        }
        published = r_end;
    }
    const Clock::time_point tw = Clock::now();
    while (cudaStreamQuery(s) == cudaErrorNotReady) {
        if (std::chrono::duration<double>(Clock::now() - tw).count() > wait_s) {
            failed = true;
            break;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    cudaStreamSynchronize(s);
    for (cudaEvent_t ev : events) cudaEventDestroy(ev);
    cudaStreamDestroy(s);
    double last = 0.0;
    int completed = 0;
    for (int r = 0; r < R; ++r) {
        if (done_s[size_t(r)] < 0.0) {
            latency_out[r] = std::nan("");
            continue;
        }
        ++completed;
        latency_out[r] = done_s[size_t(r)] - arrival_s[r];
        last = std::max(last, done_s[size_t(r)]);
    }
    report[0] = last;
    report[1] = double(stalls);
    report[2] = double(failed);
    report[3] = double(batches);
    report[4] = double(completed);
    report[5] = double(arena_floats) * 4.0;
    return (failed || completed != R) ? POLAR_ETIMEOUT : 0;
}
