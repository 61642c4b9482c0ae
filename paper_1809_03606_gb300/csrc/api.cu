// api.cu - the C ABI of polarscs.h: argument checks, device copies of plans,
// and the host-pointer convenience calls.  Every decode and encode step runs
// in the kernels of scs_decode.cu and encode.cu; nothing here computes on
// the host except argument validation and table building.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <new>
#include <cstring>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "plan.h"

namespace polarscs {

int launch_scs_decode(const polar_plan *p, const DeviceTables *dt, const float *d_llr, int B, int D, int L,
                      uint32_t *d_info, float *d_pm, int8_t *d_status, uint32_t *d_stats, cudaStream_t stream);
int launch_polar_encode(const polar_plan *p, const DeviceTables *dt, const uint32_t *d_msg, int B, uint32_t *d_cw,
                        cudaStream_t stream);
int launch_scs_decode_noalloc(const polar_plan *p, const float *d_llr, int B, int D, int L, uint32_t *d_info,
                              float *d_pm, int8_t *d_status, uint32_t *d_stats, cudaStream_t stream);
int launch_scs_decode_mixed(const polar_plan_set *set, const int4 *d_frames, const int *d_order, int B, int Dmax,
                            const float *d_llr, const long long *d_llr_off, uint32_t *d_info,
                            const long long *d_info_off, float *d_pm, int8_t *d_status, uint32_t *d_stats,
                            cudaStream_t stream, int wpb_req, int chunk_req, int nframes);
void free_set_device(polar_plan_set *set);
template <typename T>
int launch_gsc(const polar_plan *p, const uint8_t *d_info_mask, const T *d_llr, const uint32_t *d_u, int B,
               const T *d_scales, T *d_loss, T *d_grad_scales, T *d_grad_llr, T *d_leaf, cudaStream_t stream);

TraceRange::TraceRange(const char *name) { nvtxRangePushA(name); }
TraceRange::~TraceRange() { nvtxRangePop(); }

// Per-call scratch comes from the device's default stream-ordered pool.  By
// default that pool returns memory to the driver at every synchronisation,
// which would turn each call's scratch into a fresh allocation; keep it.
void keep_pool_memory(int dev) {
    static std::atomic<unsigned long long> done{0ull};
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load() & bit) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        unsigned long long thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done.fetch_or(bit);
}

int cuda_status(int err) {
    const cudaError_t e = cudaError_t(err);
    if (e == cudaSuccess) return 0;
    cudaGetLastError();  // clear a sticky non-fatal error state
    return e == cudaErrorMemoryAllocation ? POLAR_ENOMEM : POLAR_ECUDA;
}

template <typename T>
static cudaError_t upload(T **dst, const std::vector<T> &src) {
    *dst = nullptr;
    if (src.empty()) return cudaSuccess;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(dst), src.size() * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

static void free_tables(DeviceTables &d) {
    cudaFree(d.ops);
    cudaFree(d.crc_rows);
    cudaFree(d.msg_pos);
    cudaFree(d.info_pos);
    cudaFree(d.crc_contrib);
    cudaFree(d.info_mask);
    cudaFree(d.info_bits);
    cudaFree(d.scales);
    d = DeviceTables{};
}

int plan_device(const polar_plan *p, const DeviceTables **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    std::lock_guard<std::mutex> g(p->mu);
    if (p->dev.device == dev) {
        *out = &p->dev;
        return 0;
    }
    if (p->dev.device >= 0) return POLAR_EINVAL;  // a plan serves one device
    DeviceTables d{};
    d.device = dev;
    e = upload(&d.ops, p->dev_ops);
    if (e == cudaSuccess) e = upload(&d.crc_rows, p->crc_rows);
    if (e == cudaSuccess) e = upload(&d.msg_pos, p->msg_pos);
    if (e == cudaSuccess) e = upload(&d.info_pos, p->info_pos);
    if (e == cudaSuccess) e = upload(&d.crc_contrib, p->crc_contrib);
    if (e == cudaSuccess) e = upload(&d.info_mask, p->info_mask);
    if (e == cudaSuccess) e = upload(&d.info_bits, p->info_bits);
    if (e == cudaSuccess) e = upload(&d.scales, p->scales);
    if (e != cudaSuccess) {
        free_tables(d);
        return cuda_status(e);
    }
    p->dev = d;
    *out = &p->dev;
    return 0;
}

}  // namespace polarscs

using namespace polarscs;

extern "C" void polar_plan_destroy(polar_plan *p) {
    if (!p) return;
    if (p->dev.device >= 0) {
        int cur = -1;
        cudaGetDevice(&cur);
        cudaSetDevice(p->dev.device);
        free_tables(p->dev);
        if (cur >= 0) cudaSetDevice(cur);
    }
    delete p;
}

extern "C" int polar_plan_set_scales(polar_plan *p, const float *scales) {
    if (!p) return POLAR_EINVAL;
    std::lock_guard<std::mutex> g(p->mu);
    if (scales && p->exact) return POLAR_EINVAL;  // scales are a min-sum form
    if (scales) {
        for (int i = 0; i < p->n; ++i)
            if (!(scales[i] == scales[i]) || scales[i] > 3.0e38f || scales[i] < -3.0e38f) return POLAR_EINVAL;
        p->scales.assign(scales, scales + p->n);
    } else {
        p->scales.clear();
    }
    ++p->version;
    if (p->dev.device < 0) return 0;  // the device copy is made on first use
    int cur = -1;
    cudaGetDevice(&cur);
    cudaError_t e = cudaSetDevice(p->dev.device);
    if (e == cudaSuccess && !p->scales.empty() && !p->dev.scales)
        e = cudaMalloc(reinterpret_cast<void **>(&p->dev.scales), sizeof(float) * size_t(p->n));
    if (e == cudaSuccess && !p->scales.empty())
        e = cudaMemcpy(p->dev.scales, p->scales.data(), sizeof(float) * size_t(p->n), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && p->scales.empty() && p->dev.scales) {
        e = cudaFree(p->dev.scales);
        p->dev.scales = nullptr;
    }
    if (cur >= 0) cudaSetDevice(cur);
    return e == cudaSuccess ? 0 : cuda_status(e);
}

extern "C" int scs_decode_batch(const polar_plan *p, const float *d_llr, int B, int D, int L, uint32_t *d_info,
                                float *d_pm, int8_t *d_status, uint32_t *d_stats, void *stream) {
    TraceRange trace("scs_decode_batch");
    if (!p || B < 0 || D < 1 || L < 1) return POLAR_EINVAL;
    if (B > 0 && (!d_llr || !d_info || !d_pm || !d_status)) return POLAR_EINVAL;
    if (p->N > POLAR_MAX_N_GPU || D > POLAR_MAX_D_GPU_DEEP || L > POLAR_MAX_L_GPU) return POLAR_ELIMIT;
    if (D > POLAR_MAX_D_GPU && p->exact) return POLAR_ELIMIT;  // the memory stack decodes min-sum plans
    if (B == 0) return 0;
    const DeviceTables *dt = nullptr;
    int rc = plan_device(p, &dt);
    if (rc) return rc;
    return launch_scs_decode(p, dt, d_llr, B, D, L, d_info, d_pm, d_status, d_stats, cudaStream_t(stream));
}

extern "C" int scs_decode_batch_noalloc(const polar_plan *p, const float *d_llr, int B, int D, int L,
                                        uint32_t *d_info, float *d_pm, int8_t *d_status, uint32_t *d_stats,
                                        void *stream) {
    TraceRange trace("scs_decode_batch_noalloc");
    if (!p || B < 0 || D < 1 || L < 1) return POLAR_EINVAL;
    if (B > 0 && (!d_llr || !d_info || !d_pm || !d_status)) return POLAR_EINVAL;
    if (p->N > POLAR_MAX_N_GPU || D > POLAR_MAX_D_GPU || L > POLAR_MAX_L_GPU) return POLAR_ELIMIT;
    if (B == 0) return 0;
    return launch_scs_decode_noalloc(p, d_llr, B, D, L, d_info, d_pm, d_status, d_stats, cudaStream_t(stream));
}

extern "C" int polar_plan_set_create(const polar_plan *const *plans, int nplans, polar_plan_set **out) {
    if (!out || !plans || nplans < 1 || nplans > 64) return POLAR_EINVAL;
    *out = nullptr;
    for (int i = 0; i < nplans; ++i) {
        if (!plans[i] || plans[i]->exact) return POLAR_EINVAL;
        if (plans[i]->N > POLAR_MAX_N_GPU) return POLAR_ELIMIT;
    }
    polar_plan_set *set = new (std::nothrow) polar_plan_set();
    if (!set) return POLAR_ENOMEM;
    for (int i = 0; i < nplans; ++i) {
        set->plans.push_back(plans[i]);
        set->Nmax = std::max(set->Nmax, plans[i]->N);
        set->Wmax = std::max(set->Wmax, plans[i]->W);
        set->nbranch_max = std::max(set->nbranch_max, plans[i]->nbranch);
    }
    *out = set;
    return 0;
}

extern "C" void polar_plan_set_destroy(polar_plan_set *set) {
    if (!set) return;
    free_set_device(set);
    delete set;
}

static int check_mixed(const polar_plan_set *set, const int32_t *d_frames, int B, int Dmax, const float *d_llr,
                       const int64_t *d_llr_off, uint32_t *d_info, const int64_t *d_info_off, float *d_pm,
                       int8_t *d_status) {
    if (!set || B < 0 || Dmax < 1) return POLAR_EINVAL;
    if (B > 0 && (!d_frames || !d_llr || !d_llr_off || !d_info || !d_info_off || !d_pm || !d_status)) return POLAR_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_frames) & 15u) != 0u) return POLAR_EINVAL;
    if (Dmax > POLAR_MAX_D_GPU) return POLAR_ELIMIT;
    return 0;
}

extern "C" int scs_decode_mixed(const polar_plan_set *set, const int32_t *d_frames, const int32_t *d_order, int B,
                                int Dmax, const float *d_llr, const int64_t *d_llr_off, uint32_t *d_info,
                                const int64_t *d_info_off, float *d_pm, int8_t *d_status, uint32_t *d_stats,
                                void *stream) {
    TraceRange trace("scs_decode_mixed");
    int rc = check_mixed(set, d_frames, B, Dmax, d_llr, d_llr_off, d_info, d_info_off, d_pm, d_status);
    if (rc || B == 0) return rc;
    return launch_scs_decode_mixed(set, reinterpret_cast<const int4 *>(d_frames), d_order, B, Dmax, d_llr,
                                   reinterpret_cast<const long long *>(d_llr_off), d_info,
                                   reinterpret_cast<const long long *>(d_info_off), d_pm, d_status, d_stats,
                                   cudaStream_t(stream), 0, 0, B);
}

// the side stream and fork/join events of scs_decode_mixed_split, one set
// per device, made on the first call there; the mutex serialises the
// enqueueing of calls that share them
namespace {
struct SplitStreams {
    bool ready = false;
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
std::mutex g_split_mu;
SplitStreams g_split[64];
}  // namespace

extern "C" int scs_decode_mixed_split(const polar_plan_set *set, const int32_t *d_frames, const int32_t *d_order,
                                      int B, int n_two, int Dmax, const float *d_llr, const int64_t *d_llr_off,
                                      uint32_t *d_info, const int64_t *d_info_off, float *d_pm, int8_t *d_status,
                                      uint32_t *d_stats, void *stream) {
    TraceRange trace("scs_decode_mixed_split");
    int rc = check_mixed(set, d_frames, B, Dmax, d_llr, d_llr_off, d_info, d_info_off, d_pm, d_status);
    if (rc || B == 0) return rc;
    if (!d_order || n_two < 0 || n_two > B || (n_two > 0 && Dmax <= 32)) return POLAR_EINVAL;
    const int4 *fr = reinterpret_cast<const int4 *>(d_frames);
    const long long *lo = reinterpret_cast<const long long *>(d_llr_off);
    const long long *io = reinterpret_cast<const long long *>(d_info_off);
    cudaStream_t s = cudaStream_t(stream);
    const int Dmax1 = std::min(Dmax, 32);
    if (n_two == 0 || n_two == B) {  // one kind of frame only: one launch
        return launch_scs_decode_mixed(set, fr, d_order, B, n_two ? Dmax : Dmax1, d_llr, lo, d_info, io, d_pm,
                                       d_status, d_stats, s, 0, 0, B);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= 64) return POLAR_EINVAL;
    std::lock_guard<std::mutex> g(g_split_mu);
    SplitStreams &ss = g_split[dev];
    if (!ss.ready) {
        e = cudaStreamCreateWithFlags(&ss.side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ss.join, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_status(e);
        ss.ready = true;
    }
    // the two-row frames (order[0, n_two)) on the side stream, the one-row
    // frames (order[n_two, B)) on the caller's stream, joined back to it
    e = cudaEventRecord(ss.fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ss.side, ss.fork, 0);
    if (e != cudaSuccess) return cuda_status(e);
    rc = launch_scs_decode_mixed(set, fr, d_order, n_two, Dmax, d_llr, lo, d_info, io, d_pm, d_status, d_stats,
                                 ss.side, 0, 0, B);
    const int rc2 = launch_scs_decode_mixed(set, fr, d_order + n_two, B - n_two, Dmax1, d_llr, lo, d_info, io, d_pm,
                                            d_status, d_stats, s, 0, 0, B);
    e = cudaEventRecord(ss.join, ss.side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ss.join, 0);
    if (rc) return rc;
    if (rc2) return rc2;
    return e == cudaSuccess ? 0 : cuda_status(e);
}

extern "C" int scs_tune_mixed(polar_plan_set *set, const int32_t *d_frames, const int32_t *d_order, int B, int Dmax,
                              const float *d_llr, const int64_t *d_llr_off, uint32_t *d_info,
                              const int64_t *d_info_off, float *d_pm, int8_t *d_status, void *stream, int *wpb_out,
                              int *chunk_out) {
    TraceRange trace("scs_tune_mixed");
    int rc = check_mixed(set, d_frames, B, Dmax, d_llr, d_llr_off, d_info, d_info_off, d_pm, d_status);
    if (rc) return rc;
    if (B == 0) return POLAR_EINVAL;
    cudaStream_t s = cudaStream_t(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_status(e);
    }
    static const int kWpb[] = {1, 2, 4};
    static const int kChunk[] = {1, 4, 16};
    float best = -1.0f;
    int bw = 4, bc = 1;
    for (int wi = 0; wi < 3 && rc == 0; ++wi) {
        for (int ci = 0; ci < 3 && rc == 0; ++ci) {
            float ms = 0.0f;
            for (int rep = 0; rep < 2 && rc == 0; ++rep) {  // first run warms up, the second is timed
                cudaEventRecord(e0, s);
                rc = launch_scs_decode_mixed(set, reinterpret_cast<const int4 *>(d_frames), d_order, B, Dmax, d_llr,
                                             reinterpret_cast<const long long *>(d_llr_off), d_info,
                                             reinterpret_cast<const long long *>(d_info_off), d_pm, d_status, nullptr,
                                             s, kWpb[wi], kChunk[ci], B);
                cudaEventRecord(e1, s);
                e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) rc = cuda_status(e);
                if (rc == 0) cudaEventElapsedTime(&ms, e0, e1);
            }
            if (rc == 0 && (best < 0.0f || ms < best)) {
                best = ms;
                bw = kWpb[wi];
                bc = kChunk[ci];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> g(set->mu);
        set->tuned_wpb = bw;
        set->tuned_chunk = bc;
    }
    if (wpb_out) *wpb_out = bw;
    if (chunk_out) *chunk_out = bc;
    return 0;
}

extern "C" int polar_plan_set_tuning(polar_plan_set *set, int warps_per_block, int frames_per_claim) {
    if (!set) return POLAR_EINVAL;
    const bool clear = warps_per_block == 0 && frames_per_claim == 0;
    const bool wpb_ok = warps_per_block == 1 || warps_per_block == 2 || warps_per_block == 4;
    if (!clear && (!wpb_ok || frames_per_claim < 1 || frames_per_claim > 1024)) return POLAR_EINVAL;
    std::lock_guard<std::mutex> g(set->mu);
    set->tuned_wpb = warps_per_block;
    set->tuned_chunk = frames_per_claim;
    return 0;
}

extern "C" int polar_plan_set_get_tuning(const polar_plan_set *set, int *warps_per_block, int *frames_per_claim) {
    if (!set || !warps_per_block || !frames_per_claim) return POLAR_EINVAL;
    std::lock_guard<std::mutex> g(set->mu);
    *warps_per_block = set->tuned_wpb;
    *frames_per_claim = set->tuned_chunk;
    return 0;
}

template <typename T>
static int gsc_call(const polar_plan *p, const T *d_llr, const uint32_t *d_u, int B, const T *d_scales, T *d_loss,
                    T *d_grad_scales, T *d_grad_llr, T *d_leaf, void *stream) {
    TraceRange trace("gsc_loss");
    if (!p || B < 1 || !d_llr || !d_u || !d_scales || !d_loss) return POLAR_EINVAL;
    const DeviceTables *dt = nullptr;
    int rc = plan_device(p, &dt);
    if (rc) return rc;
    return launch_gsc<T>(p, dt->info_mask, d_llr, d_u, B, d_scales, d_loss, d_grad_scales, d_grad_llr, d_leaf,
                         cudaStream_t(stream));
}

extern "C" int gsc_loss(const polar_plan *p, const float *d_llr, const uint32_t *d_u, int B, const float *d_scales,
                        float *d_loss, float *d_leaf, void *stream) {
    return gsc_call<float>(p, d_llr, d_u, B, d_scales, d_loss, nullptr, nullptr, d_leaf, stream);
}

extern "C" int gsc_loss_grad(const polar_plan *p, const float *d_llr, const uint32_t *d_u, int B,
                             const float *d_scales, float *d_loss, float *d_grad_scales, float *d_grad_llr,
                             void *stream) {
    if (!d_grad_scales) return POLAR_EINVAL;
    return gsc_call<float>(p, d_llr, d_u, B, d_scales, d_loss, d_grad_scales, d_grad_llr, nullptr, stream);
}

extern "C" int gsc_loss_f64(const polar_plan *p, const double *d_llr, const uint32_t *d_u, int B,
                            const double *d_scales, double *d_loss, double *d_leaf, void *stream) {
    return gsc_call<double>(p, d_llr, d_u, B, d_scales, d_loss, nullptr, nullptr, d_leaf, stream);
}

extern "C" int gsc_loss_grad_f64(const polar_plan *p, const double *d_llr, const uint32_t *d_u, int B,
                                 const double *d_scales, double *d_loss, double *d_grad_scales, double *d_grad_llr,
                                 void *stream) {
    if (!d_grad_scales) return POLAR_EINVAL;
    return gsc_call<double>(p, d_llr, d_u, B, d_scales, d_loss, d_grad_scales, d_grad_llr, nullptr, stream);
}

// Longest-first order of a mixed batch (host): frames sorted by an estimate
// of their decoding work, N * (8 + D), descending; ties keep frame order.
// Heavy frames then start first and light ones fill the end of the launch.
extern "C" int polar_mixed_order(const polar_plan_set *set, const int32_t *h_frames, int B, int32_t *h_order) {
    if (!set || B < 0 || (B > 0 && (!h_frames || !h_order))) return POLAR_EINVAL;
    std::vector<std::pair<long long, int>> key(static_cast<size_t>(B));
    for (int b = 0; b < B; ++b) {
        const int pi = h_frames[4 * size_t(b)], D = h_frames[4 * size_t(b) + 1];
        long long w = 0;
        if (pi >= 0 && pi < int(set->plans.size())) w = (long long)set->plans[size_t(pi)]->N * (8 + std::max(D, 0));
        key[size_t(b)] = {-w, b};
    }
    std::stable_sort(key.begin(), key.end());
    for (int b = 0; b < B; ++b) h_order[b] = key[size_t(b)].second;
    return 0;
}

// The claim order of scs_decode_mixed_split (host): the frames that need two
// stack rows a lane (valid descriptors with D > 32) first, then the others,
// each part longest-first like polar_mixed_order; *n_two = the first part's size.
extern "C" int polar_mixed_split_order(const polar_plan_set *set, const int32_t *h_frames, int B, int32_t *h_order,
                                       int *n_two) {
    if (!set || B < 0 || !n_two || (B > 0 && (!h_frames || !h_order))) return POLAR_EINVAL;
    std::vector<std::pair<std::pair<int, long long>, int>> key(static_cast<size_t>(B));
    int two = 0;
    for (int b = 0; b < B; ++b) {
        const int pi = h_frames[4 * size_t(b)], D = h_frames[4 * size_t(b) + 1];
        const bool ok = pi >= 0 && pi < int(set->plans.size());
        const long long w = ok ? (long long)set->plans[size_t(pi)]->N * (8 + std::max(D, 0)) : 0;
        const int part = (ok && D > 32 && D <= POLAR_MAX_D_GPU) ? 0 : 1;
        two += part == 0;
        key[size_t(b)] = {{part, -w}, b};
    }
    std::stable_sort(key.begin(), key.end());
    for (int b = 0; b < B; ++b) h_order[b] = key[size_t(b)].second;
    *n_two = two;
    return 0;
}

extern "C" int polar_encode_batch(const polar_plan *p, const uint32_t *d_msg, int B, uint32_t *d_codeword,
                                  void *stream) {
    TraceRange trace("polar_encode_batch");
    if (!p || B < 0) return POLAR_EINVAL;
    if (B > 0 && (!d_msg || !d_codeword)) return POLAR_EINVAL;
    if (B == 0) return 0;
    const DeviceTables *dt = nullptr;
    int rc = plan_device(p, &dt);
    if (rc) return rc;
    return launch_polar_encode(p, dt, d_msg, B, d_codeword, cudaStream_t(stream));
}

extern "C" int polar_encode(const uint8_t *msg, int N, int K, const uint8_t *frozen, int crc, uint8_t *codeword) {
    if (!msg || !frozen || !codeword) return POLAR_EINVAL;
    polar_plan *p = nullptr;
    int rc = polar_plan_create(N, K, frozen, 0, crc, &p);
    if (rc) return rc;
    const int mw = (p->Kmsg + 31) / 32;
    std::vector<uint32_t> hm(static_cast<size_t>(mw), 0u), hc(static_cast<size_t>(p->W), 0u);
    for (int j = 0; j < p->Kmsg; ++j)
        if (msg[j] & 1) hm[size_t(j >> 5)] |= 1u << (j & 31);
    uint32_t *dm = nullptr, *dc = nullptr;
    cudaError_t e = cudaMalloc(&dm, hm.size() * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dc, hc.size() * 4);
    if (e == cudaSuccess) e = cudaMemcpy(dm, hm.data(), hm.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        rc = polar_encode_batch(p, dm, 1, dc, nullptr);
        if (rc == 0) e = cudaMemcpy(hc.data(), dc, hc.size() * 4, cudaMemcpyDeviceToHost);
    }
    cudaFree(dm);
    cudaFree(dc);
    polar_plan_destroy(p);
    if (e != cudaSuccess) return cuda_status(e);
    if (rc) return rc;
    for (int i = 0; i < N; ++i) codeword[i] = uint8_t((hc[size_t(i >> 5)] >> (i & 31)) & 1u);
    return 0;
}

extern "C" int scs_decode(const float *llr, int N, int K, const uint8_t *frozen, int D, int L, int crc,
                          uint8_t *info_out, float *pm_out) {
    TraceRange trace("scs_decode");
    if (!llr || !frozen || !info_out || !pm_out) return POLAR_EINVAL;
    polar_plan *p = nullptr;
    int rc = polar_plan_create(N, K, frozen, 1, crc, &p);
    if (rc) return rc;
    const int iw = (p->Kmsg + 31) / 32;
    float *dl = nullptr, *dpm = nullptr;
    uint32_t *di = nullptr;
    int8_t *dst = nullptr;
    std::vector<uint32_t> hi(size_t(iw), 0u);
    int8_t status = 0;
    cudaError_t e = cudaMalloc(&dl, size_t(N) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&di, size_t(iw) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dpm, 4);
    if (e == cudaSuccess) e = cudaMalloc(&dst, 1);
    if (e == cudaSuccess) e = cudaMemcpy(dl, llr, size_t(N) * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        rc = scs_decode_batch(p, dl, 1, D, L, di, dpm, dst, nullptr, nullptr);
        if (rc == 0) e = cudaMemcpy(hi.data(), di, size_t(iw) * 4, cudaMemcpyDeviceToHost);
        if (rc == 0 && e == cudaSuccess) e = cudaMemcpy(pm_out, dpm, 4, cudaMemcpyDeviceToHost);
        if (rc == 0 && e == cudaSuccess) e = cudaMemcpy(&status, dst, 1, cudaMemcpyDeviceToHost);
    }
    cudaFree(dl);
    cudaFree(di);
    cudaFree(dpm);
    cudaFree(dst);
    const int kmsg = p->Kmsg;
    polar_plan_destroy(p);
    if (e != cudaSuccess) return cuda_status(e);
    if (rc) return rc;
    for (int j = 0; j < kmsg; ++j) info_out[j] = uint8_t((hi[size_t(j >> 5)] >> (j & 31)) & 1u);
    return int(status);
}

extern "C" int polar_device_info(int *sm_count, int *cc_major, int *cc_minor) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (sm_count) cudaDeviceGetAttribute(sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (cc_major) cudaDeviceGetAttribute(cc_major, cudaDevAttrComputeCapabilityMajor, dev);
    if (cc_minor) cudaDeviceGetAttribute(cc_minor, cudaDevAttrComputeCapabilityMinor, dev);
    return 0;
}
