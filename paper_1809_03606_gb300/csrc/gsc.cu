// gsc.cu - genie-aided SC soft decoding with per-stage min-sum scales, and
// its hand-written reverse pass.
//
// Built on the SC recursions of the paper (Eq. minsum, Eq. llrcalc): with the
// transmitted bits known, every g uses the true partial sums, so the alpha
// tree of a frame is a fixed function of its channel LLRs and of the stage
// scales s_lambda that multiply the f outputs written at stage lambda:
//   left child  = s_lambda * f(a, b),   right child = b + (1 - 2 beta) a.
// The loss is the mean over frames and information leaves of the binary
// cross-entropy of the leaf LLR L_i against the transmitted bit u_i:
//   softplus(-(1 - 2 u_i) L_i).
//
// GB300 mapping: one CTA per frame (persistent), the whole tree ((n+1) x N
// values, stage lambda at offset lambda * N) in shared memory.  Stages are
// computed layer by layer with every thread owning node pairs: the wide top
// stages by the whole block (a block barrier per stage), the stages whose
// nodes fit in one warp's segment of N/8 positions by that warp alone (warp
// synchronisation only); the reverse pass overwrites the stage values with
// their adjoints in place (a thread reads and then writes the same two parent
// positions).  Per-frame sums go to
// a [B, n+1] buffer that a second kernel reduces over frames in a fixed order,
// so results do not depend on scheduling; inside a frame each warp reduces its
// share by a shuffle tree and the warps' sums are added in warp order once per
// frame (no block barrier per stage for the sums).  Templated on the value type:
// float for training, double for gradient checks.
#include <cuda_runtime.h>

#include <cstdint>

#include "plan.h"

namespace polarscs {
namespace {

constexpr int kGscThreads = 256;

template <typename T>
struct GscArgs {
    const T *llr;        // [B, N]
    const uint32_t *u;   // [B, W] transmitted bits u (frozen positions 0)
    const uint8_t *info; // [N] 1 = information leaf
    const T *scales;     // [n]
    int B, N, n, W;
    int with_grad;       // run the reverse pass
    T *frame_sums;       // [B, n + 1]: per-frame loss sum, then d/ds_lambda sums
    T *grad_llr;         // [B, N] or null (unnormalised adjoint of the root)
    T *leaf_out;         // [B, N] or null (leaf LLRs)
};

template <typename T>
__device__ __forceinline__ T f_ms(T a, T b) {
    const T m = fabs(a) < fabs(b) ? fabs(a) : fabs(b);
    return ((a < T(0)) != (b < T(0))) ? -m : m;
}

template <typename T>
__device__ __forceinline__ T softplus(T z) {
    return z > T(0) ? z + log1p(exp(-z)) : log1p(exp(z));
}

// one node pair forward: left child s * f(x, y), right child y + (1 - 2 beta) x
template <typename T>
__device__ __forceinline__ void fwd_pair(T x, T y, uint32_t beta, T s, T &l, T &r) {
    l = s * f_ms(x, y);
    r = beta ? y - x : y + x;
}

// one node pair in reverse: adjoints gl, gr of the children give those of
// the parents (ax, ay) and the pair's share of d/ds
template <typename T>
__device__ __forceinline__ void bwd_pair(T x, T y, T gl, T gr, uint32_t beta, T s, T &gs, T &ax, T &ay) {
    gs += gl * f_ms(x, y);
    const T sx = x < T(0) ? T(-1) : T(1), sy = y < T(0) ? T(-1) : T(1);
    ax = beta ? -gr : gr;
    ay = gr;
    if (fabs(x) <= fabs(y)) ax += gl * s * sy;  // f = s * sgn(y) * x
    else ay += gl * s * sx;                     // f = s * sgn(x) * y
}

// warp sum by a shuffle tree (the full sum ends in lane 0)
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int k = 16; k >= 1; k >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, k);
    return v;
}

// LOGN > 0: the code length 2^LOGN fixed at compile time (every index shift
// and trip count a constant); LOGN = 0: any length
template <typename T, int LOGN>
__global__ void __launch_bounds__(kGscThreads, 4) gsc_kernel(GscArgs<T> a) {
    extern __shared__ __align__(16) unsigned char gsm[];
    const int N = LOGN ? (1 << LOGN) : a.N, n = LOGN ? LOGN : a.n, W = LOGN ? ((N + 31) >> 5) : a.W;
    const int half = N >> 1;
    T *tree = reinterpret_cast<T *>(gsm);                           // (n+1) * N
    uint32_t *xs = reinterpret_cast<uint32_t *>(tree + (n + 1) * N);  // (n+1) * W partial sums
    // per-warp partial sums of the frame's loss and of d/ds_lambda, reduced
    // over the warps once per frame in warp order
    constexpr int kWarps = kGscThreads / 32;
    __shared__ T wsum[16 * kWarps];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // warp w owns positions [w seg, (w+1) seg) of every stage; a stage whose
    // parent nodes fit in a segment (2^(lambda+1) <= seg) is updated by each
    // warp on its own segment (its seg/2 node pairs), with warp-level
    // synchronisation only; wider stages are shared by the block
    const int seg = N / kWarps, pseg = seg >> 1;
    const int lam_loc = seg >= 2 ? (30 - __clz(seg)) : -1;  // highest warp-local stage
    // float and 128-position segments: stages 0 and 1 take 4 positions per
    // lane, the others two adjacent node pairs per thread (each thread's one
    // share of the warp's 64 or the block's 512 pairs)
    constexpr bool kVec = sizeof(T) == 4 && LOGN == 10 && kGscThreads == 256;
    // shared-memory position of index p of stage st: in the specialised
    // kernel stages 2-5 -- the ones the two node pairs a thread takes at
    // stages 2-4 read and write -- have the 4-value groups of the second
    // 32-value half of every 64 values permuted (bits 2-4 XOR 28), so that
    // those accesses hit 32 distinct banks per half-warp; 4-value groups stay
    // whole and aligned for the vector accesses.  The stage loops are
    // unrolled, so the stage is a constant and the other stages pay nothing.
    auto sw = [](int st, int p) { return (kVec && st >= 2 && st <= 5) ? (p ^ (((p >> 5) & 1) * 28)) : p; };
    // the specialised kernel loads the next frame's LLR row into registers
    // while the current frame is computed (N / 256 values per thread)
    constexpr int kPre = LOGN ? ((1 << LOGN) + kGscThreads - 1) / kGscThreads : 1;
    T pre[kPre];
    if (LOGN && int(blockIdx.x) < a.B) {
#pragma unroll
        for (int q = 0; q < kPre; ++q) {
            const int i = tid + q * kGscThreads;
            if (i < N) pre[q] = a.llr[size_t(blockIdx.x) * N + i];
        }
    }
    for (int b = blockIdx.x; b < a.B; b += gridDim.x) {
        if (LOGN) {
            const int bn = b + int(gridDim.x);
#pragma unroll
            for (int q = 0; q < kPre; ++q) {
                const int i = tid + q * kGscThreads;
                if (i < N) {
                    tree[size_t(n) * N + i] = pre[q];
                    if (bn < a.B) pre[q] = a.llr[size_t(bn) * N + i];
                }
            }
        } else {
            const T *l = a.llr + size_t(b) * N;
            for (int i = tid; i < N; i += blockDim.x) tree[size_t(n) * N + i] = l[i];
        }
        // partial sums (warp 0): xs[lambda] = u after the encoder stages of
        // distance 1 .. 2^(lambda-1)
        if (wid == 0) {
            for (int k = lane; k < W; k += 32) xs[k] = a.u[size_t(b) * W + k];
            __syncwarp();
            for (int lam = 0; lam < n; ++lam) {
                const uint32_t *src = xs + lam * W;
                uint32_t *dst = xs + (lam + 1) * W;
                const int d = 1 << lam;
                for (int k = lane; k < W; k += 32) {
                    uint32_t x = src[k];
                    if (d < 32) {
                        const uint32_t M = d == 1 ? 0x55555555u : d == 2 ? 0x33333333u : d == 4 ? 0x0F0F0F0Fu
                                         : d == 8 ? 0x00FF00FFu : 0x0000FFFFu;
                        x ^= (x >> d) & M;
                        if (N < 32) x &= (1u << N) - 1u;
                    } else {
                        const int dw = d >> 5;
                        if (!(k & dw)) x ^= src[k + dw];
                    }
                    dst[k] = x;
                }
                __syncwarp();
            }
        }
        __syncthreads();
        // forward, stage n-1 down to 0
#pragma unroll
        for (int lam = n - 1; lam >= 0; --lam) {
            const bool loc = lam <= lam_loc;
            const int i0 = loc ? wid * pseg + lane : tid, i1 = loc ? (wid + 1) * pseg : half;
            const int st = loc ? 32 : int(blockDim.x);
            const int len = 1 << lam;
            const T s = a.scales[lam];
            const T *par = tree + size_t(lam + 1) * N;
            T *cur = tree + size_t(lam) * N;
            const uint32_t *bx = xs + lam * W;
            bool done = false;
            if constexpr (kVec) {
                if (lam <= 1) {  // two node pairs per lane in one 16-byte access
                const int p = wid * seg + 4 * lane;
                const float4 v = *reinterpret_cast<const float4 *>(par + sw(lam + 1, p));
                const uint32_t w = bx[p >> 5] >> (p & 31);
                float4 o;
                if (lam == 0) {  // pairs (p, p+1), (p+2, p+3)
                    fwd_pair<T>(v.x, v.y, w & 1u, s, o.x, o.y);
                    fwd_pair<T>(v.z, v.w, (w >> 2) & 1u, s, o.z, o.w);
                } else {  // pairs (p, p+2), (p+1, p+3)
                    fwd_pair<T>(v.x, v.z, w & 1u, s, o.x, o.z);
                    fwd_pair<T>(v.y, v.w, (w >> 1) & 1u, s, o.y, o.w);
                }
                *reinterpret_cast<float4 *>(cur + sw(lam, p)) = o;
                done = true;
                } else {  // two adjacent node pairs per thread in 8-byte accesses
                    const int i = 2 * (loc ? wid * 32 + lane : tid);
                    const int ps = (i >> lam) << (lam + 1), j = i & (len - 1);
                    const float2 x = *reinterpret_cast<const float2 *>(par + sw(lam + 1, ps + j));
                    const float2 y = *reinterpret_cast<const float2 *>(par + sw(lam + 1, ps + len + j));
                    const uint32_t w = bx[(ps + j) >> 5] >> ((ps + j) & 31);
                    float2 l, r;
                    fwd_pair<T>(x.x, y.x, w & 1u, s, l.x, r.x);
                    fwd_pair<T>(x.y, y.y, (w >> 1) & 1u, s, l.y, r.y);
                    *reinterpret_cast<float2 *>(cur + sw(lam, ps + j)) = l;
                    *reinterpret_cast<float2 *>(cur + sw(lam, ps + len + j)) = r;
                    done = true;
                }
            }
            if (!done) {
                for (int i = i0; i < i1; i += st) {
                    const int ps = (i >> lam) << (lam + 1), j = i & (len - 1);
                    const int pos = ps + j;  // the left child's true bits
                    const uint32_t beta = (bx[pos >> 5] >> (pos & 31)) & 1u;
                    fwd_pair<T>(par[ps + j], par[ps + len + j], beta, s, cur[ps + j], cur[ps + len + j]);
                }
            }
            if (loc) __syncwarp();  // the next stage reads this warp's segment only
            else __syncthreads();
        }
        // leaves (each warp on its segment when stage 0 is warp-local): loss
        // terms and the adjoint seeds in place of the leaf values
        const bool loc0 = lam_loc >= 0;
        T loss = T(0);
        for (int i = loc0 ? wid * seg + lane : tid; i < (loc0 ? (wid + 1) * seg : N); i += loc0 ? 32 : int(blockDim.x)) {
            const T L = tree[i];
            if (a.leaf_out) a.leaf_out[size_t(b) * N + i] = L;
            T adj = T(0);
            if (a.info[i]) {
                const T sg = ((xs[i >> 5] >> (i & 31)) & 1u) ? T(-1) : T(1);  // xs[0] = u
                const T z = -sg * L;
                loss += softplus(z);
                adj = -sg / (T(1) + exp(-z));  // d softplus(z) / dL
            }
            if (a.with_grad) tree[i] = adj;
        }
        loss = warp_sum(loss);
        if (lane == 0) wsum[wid] = loss;
        if (a.with_grad) {
            if (loc0) __syncwarp();
            else __syncthreads();
#pragma unroll
            for (int lam = 0; lam < n; ++lam) {
                const bool loc = lam <= lam_loc;
                const int i0 = loc ? wid * pseg + lane : tid, i1 = loc ? (wid + 1) * pseg : half;
                const int st = loc ? 32 : int(blockDim.x);
                const int len = 1 << lam;
                const T s = a.scales[lam];
                T *par = tree + size_t(lam + 1) * N;
                const T *cur = tree + size_t(lam) * N;
                const uint32_t *bx = xs + lam * W;
                T gs = T(0);
                bool done = false;
                if constexpr (kVec) {
                    if (lam <= 1) {  // two node pairs per lane in 16-byte accesses
                    const int p = wid * seg + 4 * lane;
                    const float4 v = *reinterpret_cast<const float4 *>(par + sw(lam + 1, p));
                    const float4 c = *reinterpret_cast<const float4 *>(cur + sw(lam, p));
                    const uint32_t w = bx[p >> 5] >> (p & 31);
                    float4 o;
                    if (lam == 0) {
                        bwd_pair<T>(v.x, v.y, c.x, c.y, w & 1u, s, gs, o.x, o.y);
                        bwd_pair<T>(v.z, v.w, c.z, c.w, (w >> 2) & 1u, s, gs, o.z, o.w);
                    } else {
                        bwd_pair<T>(v.x, v.z, c.x, c.z, w & 1u, s, gs, o.x, o.z);
                        bwd_pair<T>(v.y, v.w, c.y, c.w, (w >> 1) & 1u, s, gs, o.y, o.w);
                    }
                    *reinterpret_cast<float4 *>(par + sw(lam + 1, p)) = o;
                    done = true;
                    } else {  // two adjacent node pairs per thread in 8-byte accesses
                        const int i = 2 * (loc ? wid * 32 + lane : tid);
                        const int ps = (i >> lam) << (lam + 1), j = i & (len - 1);
                        const float2 x = *reinterpret_cast<const float2 *>(par + sw(lam + 1, ps + j));
                        const float2 y = *reinterpret_cast<const float2 *>(par + sw(lam + 1, ps + len + j));
                        const float2 gl = *reinterpret_cast<const float2 *>(cur + sw(lam, ps + j));
                        const float2 gr = *reinterpret_cast<const float2 *>(cur + sw(lam, ps + len + j));
                        const uint32_t w = bx[(ps + j) >> 5] >> ((ps + j) & 31);
                        float2 ax, ay;
                        bwd_pair<T>(x.x, y.x, gl.x, gr.x, w & 1u, s, gs, ax.x, ay.x);
                        bwd_pair<T>(x.y, y.y, gl.y, gr.y, (w >> 1) & 1u, s, gs, ax.y, ay.y);
                        *reinterpret_cast<float2 *>(par + sw(lam + 1, ps + j)) = ax;
                        *reinterpret_cast<float2 *>(par + sw(lam + 1, ps + len + j)) = ay;
                        done = true;
                    }
                }
                if (!done) {
                    for (int i = i0; i < i1; i += st) {
                        const int ps = (i >> lam) << (lam + 1), j = i & (len - 1);
                        const int pos = ps + j;
                        const uint32_t beta = (bx[pos >> 5] >> (pos & 31)) & 1u;
                        T ax, ay;
                        bwd_pair<T>(par[ps + j], par[ps + len + j], cur[ps + j], cur[ps + len + j], beta, s, gs, ax, ay);
                        par[ps + j] = ax;
                        par[ps + len + j] = ay;
                    }
                }
                gs = warp_sum(gs);
                if (lane == 0) wsum[(1 + lam) * kWarps + wid] = gs;
                if (lam + 1 <= lam_loc) __syncwarp();  // the next stage is this warp's too
                else __syncthreads();
            }
            if (a.grad_llr)
                for (int i = tid; i < N; i += blockDim.x) a.grad_llr[size_t(b) * N + i] = tree[size_t(n) * N + i];
        }
        __syncthreads();
        const int nq = a.with_grad ? n + 1 : 1;
        if (tid < nq) {
            T sum = T(0);
            for (int i = 0; i < kWarps; ++i) sum += wsum[tid * kWarps + i];
            a.frame_sums[size_t(b) * (n + 1) + tid] = sum;
        }
        __syncthreads();
    }
}

// out[q] = norm * sum_b frame_sums[b, q] in a fixed order (double accumulators)
template <typename T>
__global__ void gsc_reduce_kernel(const T *frame_sums, int B, int Q, double norm, T *out) {
    __shared__ double part[256];
    const int q = blockIdx.x;
    double acc = 0.0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) acc += double(frame_sums[size_t(b) * Q + q]);
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int h = blockDim.x >> 1; h >= 1; h >>= 1) {
        if (int(threadIdx.x) < h) part[threadIdx.x] += part[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = T(part[0] * norm);
}

template <typename T>
__global__ void scale_kernel(T *x, size_t n, double s) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        x[i] = T(double(x[i]) * s);
}

}  // namespace

int gsc_smem_bytes(int N, int n, int W, int elem) { return (n + 1) * N * elem + (n + 1) * W * 4; }

template <typename T>
int launch_gsc(const polar_plan *p, const uint8_t *d_info_mask, const T *d_llr, const uint32_t *d_u, int B,
               const T *d_scales, T *d_loss, T *d_grad_scales, T *d_grad_llr, T *d_leaf, cudaStream_t stream) {
    const int N = p->N, n = p->n, W = p->W;
    const int smem = gsc_smem_bytes(N, n, W, int(sizeof(T)));
    int dev = 0, sms = 0, max_smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem + int(33 * sizeof(T)) > max_smem) return POLAR_ELIMIT;
    void (*kern)(GscArgs<T>) = N == 1024 ? gsc_kernel<T, 10> : gsc_kernel<T, 0>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_status(e);
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGscThreads, smem);
    if (e != cudaSuccess) return cuda_status(e);
    if (per_sm < 1) return POLAR_ELIMIT;
    long long grid = (long long)sms * per_sm;
    if (grid > B) grid = B;
    const int Q = n + 1;
    void *ws = nullptr;
    keep_pool_memory(dev);
    e = cudaMallocAsync(&ws, size_t(B) * Q * sizeof(T) + sizeof(T) * Q, stream);
    if (e != cudaSuccess) return cuda_status(e);
    T *sums = static_cast<T *>(ws);
    T *red = sums + size_t(B) * Q;
    const bool grad = d_grad_scales != nullptr || d_grad_llr != nullptr;
    GscArgs<T> a{d_llr, d_u, d_info_mask, d_scales, B, N, n, W, grad ? 1 : 0, sums, d_grad_llr, d_leaf};
    kern<<<unsigned(grid), kGscThreads, size_t(smem), stream>>>(a);
    e = cudaGetLastError();
    int K = 0;
    for (int i = 0; i < N; ++i) K += p->frozen[size_t(i)] ? 0 : 1;
    const double norm = 1.0 / (double(B) * double(K));
    if (e == cudaSuccess) {
        gsc_reduce_kernel<T><<<unsigned(Q), 256, 0, stream>>>(sums, B, Q, norm, red);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && d_loss) e = cudaMemcpyAsync(d_loss, red, sizeof(T), cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess && d_grad_scales)
        e = cudaMemcpyAsync(d_grad_scales, red + 1, sizeof(T) * n, cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess && d_grad_llr) {
        scale_kernel<T><<<unsigned(sms > 0 ? sms * 4 : 64), 256, 0, stream>>>(d_grad_llr, size_t(B) * N, norm);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaFreeAsync(ws, stream);
    if (e != cudaSuccess) return cuda_status(e);
    return e2 == cudaSuccess ? 0 : cuda_status(e2);
}

template int launch_gsc<float>(const polar_plan *, const uint8_t *, const float *, const uint32_t *, int, const float *,
                               float *, float *, float *, float *, cudaStream_t);
template int launch_gsc<double>(const polar_plan *, const uint8_t *, const double *, const uint32_t *, int,
                                const double *, double *, double *, double *, double *, cudaStream_t);

}  // namespace polarscs
