// scs_decode.cu - FSSCS-RM stack decoding of many independent frames on
// sm_103a (Sec. 2.2.5 SCS, Sec. 3.3 reduced memory, Sec. 4 fast simplified
// stack decoding).
//
// GB300 mapping
//  - One warp decodes one frame; warps are persistent and claim frames from
//    a global counter, so frames of very different cost (path switches grow
//    at low SNR) balance across the 152 SMs.
//  - Per warp, shared memory holds the single alpha tree of the reduced-
//    memory scheme (stage lambda at float offset 2^lambda, the root stays in
//    global memory and is read through L2), the in-place N-bit beta array
//    (packed 32 bits per word) and the per-node visit counters.
//  - The stack (D <= 64 entries) lives in registers, one entry per lane for
//    D <= 32 and two for D <= 64: path metric bits, length|schedule
//    position, sequence number and a reference to a beta snapshot plus a
//    flip mask.  Pop, worst-entry search and the L-prune are warp reductions
//    (redux.sync).  Deeper stacks (up to 65536 entries, e.g. D = 8192 of
//    Sec. 5) keep the same records in per-warp scratch memory with the best
//    entry of every block of 32 in shared memory (MemStack below).
//  - Each branching node writes ONE snapshot of the beta array (the hard
//    decisions of the node in place) to scratch global memory; its 2-8
//    candidates differ from it by flips of at most 4 positions (or all
//    positions for REP), so a candidate costs registers only.  Snapshots are
//    read back only on a path switch, after which the alpha spine is
//    recomputed from the channel LLRs (Alg. calp).
//  - The decode loop is kept small.  The warps of an SM sit in different
//    parts of it and instruction fetch is their most frequent stall, so the
//    lane-strided data loops are not unrolled and the rare paths (nodes wider
//    than a warp, the restore after a path switch, CRC and output) are out of
//    line.
//  - All arithmetic on alpha and path metrics is float32 add/min/compare in
//    the order of the reference definitions; the only products are the
//    optional per-stage scales of f, rounded on their own (no FMA).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "plan.h"

namespace polarscs {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr uint32_t EMPTY = 0xFFFFFFFFu;  // path-metric bits of an empty slot
constexpr uint32_t NOSNAP = 0xFFu;       // snapshot id of the initial path
constexpr uint32_t NOSNAP_DEEP = 0xFFFFFFu;  // the same for the memory stack (24-bit slot ids)
constexpr uint32_t FLIP_ALL = 16u;       // REP second candidate: flip every bit
// SPC candidates (reading R8): the 8 flip masks over the four least reliable
// positions whose parity equals the hard-decision parity, ascending, packed
// one 4-bit mask per nibble
constexpr uint32_t SPC_MASKS_EVEN = 0xFCA96530u;  // 0,3,5,6,9,10,12,15
constexpr uint32_t SPC_MASKS_ODD = 0xEDB87421u;   // 1,2,4,7,8,11,13,14
constexpr uint32_t R1_MASKS = 0x3210u;            // Chase-II: none, m1, m2, both
constexpr uint32_t LEAF1_MASKS = 0x10u;           // decision, flipped decision

// One polar code as the kernel sees it: its schedule and tables (device
// pointers) and sizes.
struct Code {
    const KOp *ops;
    const uint32_t *crc_rows;
    const uint16_t *msg_pos;
    const float *scales;  // per-stage factors on f outputs, or null
    int N, n, W, Kmsg, crc, nops, nbranch, info_words;
    int snap_words;  // words per snapshot slot: W beta words + 4 meta words, padded
    int systematic;  // message bits read straight from the codeword estimate
};

// bytes of a plan set's code table (at most 64 codes) at the front of a mixed
// or served launch's dynamic shared memory: sized by the set's codes, not by
// the largest set, so that a set of large codes keeps one more block per SM
// (e.g. 25 codes up to N = 2048: 6 blocks of 4 warps fit, against 5 with a
// 64-entry table)
int codes_smem_bytes(int ncodes) { return (int(sizeof(Code)) * ncodes + 15) & ~15; }
// scratch budget of one memory-stack launch (D > 64): fewer resident warps
// when one warp's snapshots and entries are large
constexpr long long kDeepScratchBytes = 8LL << 30;
constexpr int kBadFrame = 3;   // status of a mixed-batch frame whose descriptor is invalid

struct Args {
    Code code;                  // uniform batch: every frame uses this code, D and L
    int D, L;
    const Code *codes;          // mixed batch: frame b uses codes[frames[b].x]
    int ncodes;
    const int4 *frames;         // mixed: (code index, D, L, unused) per frame
    const int *order;           // mixed: claim k decodes frame order[k] (null: k)
    int nframes;                // mixed: frames of the whole batch (order entries below it are decoded)
    const long long *llr_off;   // mixed: index of frame b's first LLR
    const long long *info_off;  // mixed: index of frame b's first message word
    int Dmax;                   // mixed: largest D the scratch was sized for
    const float *llr;
    int B;
    uint32_t *info_out;
    float *pm_out;
    int8_t *status_out;
    uint32_t *stats_out;
    uint32_t *scratch;
    long long scratch_stride;   // snapshot words per warp
    unsigned *counter;
    int warp_smem;              // bytes of shared memory per warp
    int codes_smem;             // mixed / served: bytes of the code table before the warps' areas
    int llr_vec;                // the LLR buffer is 16-byte aligned
    int chunk;                  // frames claimed per atomic
    // served mode: requests become decodable when the host publishes them
    const unsigned long long *head;  // device: requests [0, head) are published
    const int *abort_flag;           // host-mapped: stop waiting
    unsigned char *done_flag;        // host-mapped: 1 when request k is complete
    unsigned long long *t_done;      // device: %globaltimer at completion
    unsigned long long *t_start;     // device: %globaltimer when a warp starts the request
    int *error_flag;                 // device: a wait ran out
    unsigned long long wait_ns;      // longest wait for one request
    long long serve_stage_off;       // words into a warp's scratch where its LLR staging starts
    // memory stack (D > 64): entries after the snapshots in a warp's scratch,
    // per-block best entries after the visit counters in its shared memory
    long long deep_ent_off;          // words into a warp's scratch
    int deep_best_off;               // bytes into a warp's shared memory
    int deep_cap;                    // entries the region holds
};

// Optional per-phase cycle counters (debug builds with -DPOLAR_PHASE_TIMERS):
// lane 0 of every warp adds clock64() deltas per phase of the search into a
// device array read back by polar_phase_cycles().  Off by default.
enum Phase { PH_POP, PH_BETA, PH_ALPHA, PH_FG, PH_COMB, PH_R0, PH_NODE, PH_SNAP, PH_INSERT, PH_PRUNE, PH_DONE, PH_OUT, PH_N };
#ifdef POLAR_PHASE_TIMERS
__device__ unsigned long long g_phase_cycles[PH_N];
#define PT_INIT long long pt_t = clock64(); unsigned long long pt_acc[PH_N] = {};
#define PT(ph) { const long long pt_n = clock64(); pt_acc[ph] += (unsigned long long)(pt_n - pt_t); pt_t = pt_n; }
#define PT_FLUSH if (lane == 0) { for (int q = 0; q < PH_N; ++q) atomicAdd(&g_phase_cycles[q], pt_acc[q]); }
#else
#define PT_INIT
#define PT(ph)
#define PT_FLUSH
#endif

// POLAR_DEBUG builds check the indices of the shared-memory tree, the beta
// array, the visit counters, the snapshots and the message positions before
// they are used; a failed check skips the access and marks the frame, whose
// status becomes POLAR_DEBUG_FAIL.  Other builds compile the checks away.
#ifdef POLAR_DEBUG
#define PCK(c) ((c) ? true : (bad = 1, false))
#else
#define PCK(c) true
#endif

__device__ __forceinline__ float f_minsum(float a, float b) {
    // Eq. minsum: sign(a) sign(b) min(|a|, |b|); the sign bit is the XOR of
    // the operands' sign bits
    const float m = fminf(fabsf(a), fabsf(b));
    const uint32_t sg = (__float_as_uint(a) ^ __float_as_uint(b)) & 0x80000000u;
    return __uint_as_float(__float_as_uint(m) | sg);
}

// Eq. minsum / Fig. minsum: g = b + (1 - 2 beta) a, a = alpha_p[i],
// b = alpha_p[i + Lambda].  b + (-a) is b - a exactly in IEEE arithmetic.
__device__ __forceinline__ float g_op(float a, float b, uint32_t bit) {
    return __fadd_rn(b, __uint_as_float(__float_as_uint(a) ^ (bit << 31)));
}

// ln(1 + e^x), written so that neither branch overflows
__device__ __forceinline__ float softplus_f(float x) {
    return x > 0.0f ? __fadd_rn(x, log1pf(expf(-x))) : log1pf(expf(x));
}

// the box-plus f of Eq. llrcalc itself, 2 atanh(tanh(a/2) tanh(b/2)), as
// sgn(a) sgn(b) min(|a|,|b|) + ln(1 + e^-|a+b|) - ln(1 + e^-|a-b|), summed
// left to right (exact-f decoding)
__device__ __forceinline__ float f_exact(float a, float b) {
    const float m = fminf(fabsf(a), fabsf(b));
    const float s = ((a < 0.0f) != (b < 0.0f)) ? -m : m;
    return __fsub_rn(__fadd_rn(s, log1pf(expf(-fabsf(__fadd_rn(a, b))))), log1pf(expf(-fabsf(__fsub_rn(a, b)))));
}

__device__ __forceinline__ float pen_transform(float x, int mode) {
    // 0: x; 1: |x| where HD(x) = 1 (disagrees with 0); 2: |x| where HD(x) = 0;
    // 3: ln(1 + e^-x), the exact metric of a leaf decided 0
    if (mode == 0) return x;
    if (mode == 3) return softplus_f(-x);
    const bool neg = x < 0.0f;
    return (mode == 1) == neg ? fabsf(x) : 0.0f;
}

// Node reductions over more than 32 values (the few Rate-0, REP, Rate-1 and
// SPC nodes above stage 5): out of line, so that the per-op code the warps
// share stays small.

// sum of the node's values (transformed by `mode`) in halving order; levels
// wider than a warp are written into the free alpha stages below the node
__device__ __noinline__ float node_sum_wide(float *alpha, const float *A, int len, int mode, int lane) {
    int h = len >> 1;
    float *dst = alpha + h;
    #pragma unroll 1
    for (int i = lane; i < h; i += 32) dst[i] = __fadd_rn(pen_transform(A[i], mode), pen_transform(A[i + h], mode));
    __syncwarp();
    const float *src = dst;
    while (h > 32) {
        h >>= 1;
        float *d2 = alpha + h;
        #pragma unroll 1
        for (int i = lane; i < h; i += 32) d2[i] = __fadd_rn(src[i], src[i + h]);
        __syncwarp();
        src = d2;
    }
    float v = src[lane];
    __syncwarp();
    for (int k = 16; k >= 1; k >>= 1) {
        const float o = __shfl_down_sync(FULL, v, k);
        if (lane < k) v = __fadd_rn(v, o);
    }
    return __shfl_sync(FULL, v, 0);
}

// Loads of the channel LLRs and of beta snapshots: through L2 only (CG) or
// the default path through L1.  A frame's LLR row and its snapshots are read
// again, if at all, long after L1 has dropped them, so the register-stack
// decoders load them through L2 and keep L1 for their spilled registers
// (sweep +1.1 %, mixed batch +3 %); the memory-stack decoder measured 4 %
// slower that way and keeps the default path.
template <bool CG, class T>
__device__ __forceinline__ T ld_l2(const T *p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// path switch: the popped path's beta from its snapshot (the node's hard
// decisions) with its flips applied; returns the first bit position where
// it may differ from the beta it replaces (out of line)
__device__ __noinline__ int restore_switch(const uint32_t *sp, uint32_t *beta, int W, uint32_t mask, int lane) {
    const uint32_t m01 = sp[W], m23 = sp[W + 1];
    const int ss = int(sp[W + 2]), slam = int(sp[W + 3]);
    uint32_t dl = EMPTY;
    #pragma unroll 1
    for (int k = lane; k < W; k += 32) {
        const uint32_t nv = sp[k];
        const uint32_t x = nv ^ beta[k];
        beta[k] = nv;
        if (x && dl == EMPTY) dl = uint32_t(32 * k + __ffs(x) - 1);
    }
    dl = __reduce_min_sync(FULL, dl);
    __syncwarp();
    if (mask & FLIP_ALL) {
        const int len = 1 << slam;
        if (len >= 32) {
            #pragma unroll 1
            for (int k = lane; k < (len >> 5); k += 32) beta[(ss >> 5) + k] ^= FULL;
        } else if (lane == 0) {
            beta[ss >> 5] ^= ((1u << len) - 1u) << (ss & 31);
        }
    }
    if (lane == 0) {
        const int mm[4] = {int(m01 & 0xFFFFu), int(m01 >> 16), int(m23 & 0xFFFFu), int(m23 >> 16)};
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if ((mask >> j) & 1u) {
                const int pos = ss + mm[j];
                beta[pos >> 5] ^= 1u << (pos & 31);
            }
    }
    __syncwarp();
    return int(min(dl, uint32_t(ss)));  // the flips only touch [ss, ...)
}

// restore_switch, f_root and g_root with their global loads through L2 only
// (the register-stack decoders).  Separate copies: with one template body
// shared by both forms the memory-stack decoder, which runs the originals,
// measured 2.6 % slower with the same registers and no spills.
__device__ __noinline__ int restore_switch_cg(const uint32_t *sp, uint32_t *beta, int W, uint32_t mask, int lane) {
    const uint32_t m01 = __ldcg(sp + W), m23 = __ldcg(sp + W + 1);
    const int ss = int(__ldcg(sp + W + 2)), slam = int(__ldcg(sp + W + 3));
    uint32_t dl = EMPTY;
    #pragma unroll 1
    for (int k = lane; k < W; k += 32) {
        const uint32_t nv = __ldcg(sp + k);
        const uint32_t x = nv ^ beta[k];
        beta[k] = nv;
        if (x && dl == EMPTY) dl = uint32_t(32 * k + __ffs(x) - 1);
    }
    dl = __reduce_min_sync(FULL, dl);
    __syncwarp();
    if (mask & FLIP_ALL) {
        const int len = 1 << slam;
        if (len >= 32) {
            #pragma unroll 1
            for (int k = lane; k < (len >> 5); k += 32) beta[(ss >> 5) + k] ^= FULL;
        } else if (lane == 0) {
            beta[ss >> 5] ^= ((1u << len) - 1u) << (ss & 31);
        }
    }
    if (lane == 0) {
        const int mm[4] = {int(m01 & 0xFFFFu), int(m01 >> 16), int(m23 & 0xFFFFu), int(m23 >> 16)};
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if ((mask >> j) & 1u) {
                const int pos = ss + mm[j];
                beta[pos >> 5] ^= 1u << (pos & 31);
            }
    }
    __syncwarp();
    return int(min(dl, uint32_t(ss)));  // the flips only touch [ss, ...)
}

// f and g from the channel LLRs (the root stage, in global memory), out of
// line: vector loads when the rows are 16-byte aligned
__device__ __noinline__ void f_root(const float *P, float *C, int len, float sv, int vec, int exact, int lane) {
    if (exact) {
        #pragma unroll 1
        for (int i = lane; i < len; i += 32) C[i] = f_exact(P[i], P[i + len]);
    } else if (vec && len >= 128) {
        #pragma unroll 1
        for (int i = 4 * lane; i < len; i += 128) {
            const float4 x = *reinterpret_cast<const float4 *>(P + i);
            const float4 y = *reinterpret_cast<const float4 *>(P + i + len);
            float4 r;
            r.x = __fmul_rn(sv, f_minsum(x.x, y.x));
            r.y = __fmul_rn(sv, f_minsum(x.y, y.y));
            r.z = __fmul_rn(sv, f_minsum(x.z, y.z));
            r.w = __fmul_rn(sv, f_minsum(x.w, y.w));
            *reinterpret_cast<float4 *>(C + i) = r;
        }
    } else {
        #pragma unroll 1
        for (int i = lane; i < len; i += 32) C[i] = __fmul_rn(sv, f_minsum(P[i], P[i + len]));
    }
}

__device__ __noinline__ void g_root(const float *P, float *C, const uint32_t *beta, int len, int sl, int vec,
                                    int lane) {
    if (vec && len >= 128) {
        #pragma unroll 1
        for (int i = 4 * lane; i < len; i += 128) {
            const int pos = sl + i;
            const uint32_t bits = beta[pos >> 5] >> (pos & 31);
            const float4 x = *reinterpret_cast<const float4 *>(P + i);
            const float4 y = *reinterpret_cast<const float4 *>(P + i + len);
            float4 r;
            r.x = g_op(x.x, y.x, bits & 1u);
            r.y = g_op(x.y, y.y, (bits >> 1) & 1u);
            r.z = g_op(x.z, y.z, (bits >> 2) & 1u);
            r.w = g_op(x.w, y.w, (bits >> 3) & 1u);
            *reinterpret_cast<float4 *>(C + i) = r;
        }
    } else {
        #pragma unroll 1
        for (int i = lane; i < len; i += 32) {
            const int pos = sl + i;
            const uint32_t bit = (beta[pos >> 5] >> (pos & 31)) & 1u;
            C[i] = g_op(P[i], P[i + len], bit);
        }
    }
}

__device__ __noinline__ void f_root_cg(const float *P, float *C, int len, float sv, int vec, int exact, int lane) {
    if (exact) {
        #pragma unroll 1
        for (int i = lane; i < len; i += 32) C[i] = f_exact(__ldcg(P + i), __ldcg(P + i + len));
    } else if (vec && len >= 128) {
        #pragma unroll 1
        for (int i = 4 * lane; i < len; i += 128) {
            const float4 x = __ldcg(reinterpret_cast<const float4 *>(P + i));
            const float4 y = __ldcg(reinterpret_cast<const float4 *>(P + i + len));
            float4 r;
            r.x = __fmul_rn(sv, f_minsum(x.x, y.x));
            r.y = __fmul_rn(sv, f_minsum(x.y, y.y));
            r.z = __fmul_rn(sv, f_minsum(x.z, y.z));
            r.w = __fmul_rn(sv, f_minsum(x.w, y.w));
            *reinterpret_cast<float4 *>(C + i) = r;
        }
    } else {
        #pragma unroll 1
        for (int i = lane; i < len; i += 32) C[i] = __fmul_rn(sv, f_minsum(__ldcg(P + i), __ldcg(P + i + len)));
    }
}

__device__ __noinline__ void g_root_cg(const float *P, float *C, const uint32_t *beta, int len, int sl, int vec,
                                       int lane) {
    if (vec && len >= 128) {
        #pragma unroll 1
        for (int i = 4 * lane; i < len; i += 128) {
            const int pos = sl + i;
            const uint32_t bits = beta[pos >> 5] >> (pos & 31);
            const float4 x = __ldcg(reinterpret_cast<const float4 *>(P + i));
            const float4 y = __ldcg(reinterpret_cast<const float4 *>(P + i + len));
            float4 r;
            r.x = g_op(x.x, y.x, bits & 1u);
            r.y = g_op(x.y, y.y, (bits >> 1) & 1u);
            r.z = g_op(x.z, y.z, (bits >> 2) & 1u);
            r.w = g_op(x.w, y.w, (bits >> 3) & 1u);
            *reinterpret_cast<float4 *>(C + i) = r;
        }
    } else {
        #pragma unroll 1
        for (int i = lane; i < len; i += 32) {
            const int pos = sl + i;
            const uint32_t bit = (beta[pos >> 5] >> (pos & 31)) & 1u;
            C[i] = g_op(__ldcg(P + i), __ldcg(P + i + len), bit);
        }
    }
}

struct Least {
    int m[4];
    float mag[4];
};

// the k least reliable of `len` > 32 values (|alpha|, ties to the lower index)
__device__ __noinline__ Least node_least_wide(const float *A, int len, int k, int lane) {
    Least r{{0, 0, 0, 0}, {0.0f, 0.0f, 0.0f, 0.0f}};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (j >= k) break;
        uint32_t bv = EMPTY, bi = EMPTY;
        #pragma unroll 1
        for (int i = lane; i < len; i += 32) {
            bool used = false;
#pragma unroll
            for (int q = 0; q < 4; ++q) used |= (q < j) && (r.m[q] == i);
            if (used) continue;
            const uint32_t v = __float_as_uint(fabsf(A[i]));
            if (v < bv) {
                bv = v;
                bi = uint32_t(i);
            }
        }
        const uint32_t gv = __reduce_min_sync(FULL, bv);
        const uint32_t gi = __reduce_min_sync(FULL, bv == gv ? bi : EMPTY);
        r.m[j] = int(gi);
        r.mag[j] = __uint_as_float(gv);
    }
    return r;
}

struct Warp {
    const int lane;
    const int n;          // stage of the root
    const int llr_vec;    // the root may be read with vector loads
    float *alpha;     // shared: stage lambda at alpha + 2^lambda
    uint32_t *beta;   // shared: W words
    uint8_t *cnt;     // shared: visit counters
    uint32_t *scr;    // global: (D + 1) snapshot slots
    const float *root;
    const float *scales;  // f output scale per stage, or null (plain min-sum)
    mutable int bad;      // POLAR_DEBUG builds: an index check failed in this frame

    __device__ const float *stage(int lam) const { return lam == n ? root : alpha + (1 << lam); }
    __device__ int N() const { return 1 << n; }
    __device__ bool PCK_snap(int ss, int slam) const { return PCK(slam >= 0 && slam <= n && ss >= 0 && ss + (1 << slam) <= N()); }

    // alpha of the even child (lamc) from its parent (Eq. llrcalc, f); every
    // min-sum f output is multiplied by the stage scale (1.0, an exact
    // identity, for plain min-sum); EXACT: the box-plus f itself
    template <bool EXACT, bool CG>
    __device__ void op_f(int lamc) const {
        if (!PCK(lamc >= 0 && lamc < n)) {
            __syncwarp();
            return;
        }
        const int len = 1 << lamc;
        float *C = alpha + len;
        const float sv = scales ? __ldg(scales + lamc) : 1.0f;
        if (lamc + 1 == n) {
            (CG ? f_root_cg : f_root)(root, C, len, sv, llr_vec, EXACT ? 1 : 0, lane);
            __syncwarp();
            return;
        }
        const float *P = alpha + 2 * len;
        if (EXACT) {
            #pragma unroll 1
            for (int i = lane; i < len; i += 32) C[i] = f_exact(P[i], P[i + len]);
        } else if (len >= 128) {
            #pragma unroll 1
            for (int i = 4 * lane; i < len; i += 128) {
                const float4 x = *reinterpret_cast<const float4 *>(P + i);
                const float4 y = *reinterpret_cast<const float4 *>(P + i + len);
                float4 r;
                r.x = __fmul_rn(sv, f_minsum(x.x, y.x));
                r.y = __fmul_rn(sv, f_minsum(x.y, y.y));
                r.z = __fmul_rn(sv, f_minsum(x.z, y.z));
                r.w = __fmul_rn(sv, f_minsum(x.w, y.w));
                *reinterpret_cast<float4 *>(C + i) = r;
            }
        } else {
            #pragma unroll 1
            for (int i = lane; i < len; i += 32) C[i] = __fmul_rn(sv, f_minsum(P[i], P[i + len]));
        }
        __syncwarp();
    }

    // alpha of the odd child (lamc, sc) from its parent and the left
    // sibling's bits beta[sc - 2^lamc, sc) (Eq. llrcalc, g)
    template <bool CG>
    __device__ void op_g(int lamc, int sc) const {
        if (!PCK(lamc >= 0 && lamc < n && sc >= (1 << lamc) && sc + (1 << lamc) <= N())) {
            __syncwarp();
            return;
        }
        const int len = 1 << lamc;
        const int sl = sc - len;
        float *C = alpha + len;
        if (lamc + 1 == n) {
            (CG ? g_root_cg : g_root)(root, C, beta, len, sl, llr_vec, lane);
            __syncwarp();
            return;
        }
        const float *P = alpha + 2 * len;
        if (len >= 128) {
            #pragma unroll 1
            for (int i = 4 * lane; i < len; i += 128) {
                const int pos = sl + i;  // a multiple of 4: the 4 bits share a word
                const uint32_t bits = beta[pos >> 5] >> (pos & 31);
                const float4 x = *reinterpret_cast<const float4 *>(P + i);
                const float4 y = *reinterpret_cast<const float4 *>(P + i + len);
                float4 r;
                r.x = g_op(x.x, y.x, bits & 1u);
                r.y = g_op(x.y, y.y, (bits >> 1) & 1u);
                r.z = g_op(x.z, y.z, (bits >> 2) & 1u);
                r.w = g_op(x.w, y.w, (bits >> 3) & 1u);
                *reinterpret_cast<float4 *>(C + i) = r;
            }
        } else {
            #pragma unroll 1
            for (int i = lane; i < len; i += 32) {
                const int pos = sl + i;
                const uint32_t bit = (beta[pos >> 5] >> (pos & 31)) & 1u;
                C[i] = g_op(P[i], P[i + len], bit);
            }
        }
        __syncwarp();
    }

    // in-place beta operation of Sec. 4: beta[sl + i] ^= beta[sr + i]
    __device__ void op_comb(int lamc, int sr) const {
        if (!PCK(lamc >= 0 && lamc < n && sr >= (1 << lamc) && sr + (1 << lamc) <= N())) {
            __syncwarp();
            return;
        }
        const int len = 1 << lamc;
        const int sl = sr - len;
        if (len >= 32) {
            const int wl = sl >> 5, wr = sr >> 5, nw = len >> 5;
            #pragma unroll 1
            for (int k = lane; k < nw; k += 32) beta[wl + k] ^= beta[wr + k];
        } else if (lane == 0) {
            const int w = sl >> 5, off = sl & 31;
            const uint32_t v = beta[w];
            const uint32_t mask = ((1u << len) - 1u) << off;
            beta[w] = v ^ ((v >> len) & mask);
        }
        __syncwarp();
    }

    // set beta[s, s + 2^lam) to all-zero or all-one
    __device__ void set_range(int lam, int s, uint32_t bit) const {
        if (!PCK(lam >= 0 && lam <= n && s >= 0 && s + (1 << lam) <= N())) {
            __syncwarp();
            return;
        }
        const int len = 1 << lam;
        if (len >= 32) {
            const uint32_t v = bit ? FULL : 0u;
            #pragma unroll 1
            for (int k = lane; k < (len >> 5); k += 32) beta[(s >> 5) + k] = v;
        } else if (lane == 0) {
            const uint32_t mask = ((1u << len) - 1u) << (s & 31);
            const uint32_t w = beta[s >> 5];
            beta[s >> 5] = bit ? (w | mask) : (w & ~mask);
        }
        __syncwarp();
    }

    // ---- reductions of the node decoders over the node's alpha ----
    // hard decisions into beta[s, s + 2^lam); returns their parity (XOR)
    __device__ uint32_t node_hd(int lam, int s) const {
        if (!PCK(lam >= 0 && lam <= n && s >= 0 && s + (1 << lam) <= N())) return 0u;
        const int len = 1 << lam;
        const float *A = stage(lam);
        uint32_t par = 0;
        if (len >= 32) {
            for (int c = 0; c < (len >> 5); ++c) {
                const uint32_t bits = __ballot_sync(FULL, A[c * 32 + lane] < 0.0f);
                par ^= __popc(bits) & 1u;
                if (lane == 0) beta[(s >> 5) + c] = bits;
            }
        } else {
            const uint32_t bits = __ballot_sync(FULL, lane < len && A[lane] < 0.0f);
            par = __popc(bits) & 1u;
            if (lane == 0) {
                const uint32_t mask = ((1u << len) - 1u) << (s & 31);
                beta[s >> 5] = (beta[s >> 5] & ~mask) | (bits << (s & 31));
            }
        }
        __syncwarp();
        return par;
    }

    // sum over the node's 2^lam alpha values (transformed) in halving order:
    // v[i] += v[i + h], h = 2^(lam-1) ... 1.  Levels wider than a warp are
    // written into the free alpha stages below the node.
    __device__ float node_sum(int lam, int mode) const {
        if (!PCK(lam >= 0 && lam <= n)) return 0.0f;
        const int len = 1 << lam;
        const float *A = stage(lam);
        if (len <= 32) {
            float v = lane < len ? pen_transform(A[lane], mode) : 0.0f;
            for (int h = len >> 1; h >= 1; h >>= 1) {
                const float o = __shfl_down_sync(FULL, v, h);
                if (lane < h) v = __fadd_rn(v, o);
            }
            return __shfl_sync(FULL, v, 0);
        }
        return node_sum_wide(alpha, A, len, mode, lane);
    }

    // REP node of at most 32 values: S = sum alpha, and the penalties of the
    // all-zero and all-one words, each summed in halving order in one tree
    __device__ void rep_sums(int lam, float &S, float &pen0, float &pen1) const {
        if (!PCK(lam >= 0 && lam <= 5)) {
            S = pen0 = pen1 = 0.0f;
            return;
        }
        const int len = 1 << lam;
        const float *A = stage(lam);
        const float x = lane < len ? A[lane] : 0.0f;
        float v = x, p0 = pen_transform(x, 1), p1 = lane < len ? pen_transform(x, 2) : 0.0f;
        for (int h = len >> 1; h >= 1; h >>= 1) {
            const float ov = __shfl_down_sync(FULL, v, h);
            const float o0 = __shfl_down_sync(FULL, p0, h);
            const float o1 = __shfl_down_sync(FULL, p1, h);
            if (lane < h) {
                v = __fadd_rn(v, ov);
                p0 = __fadd_rn(p0, o0);
                p1 = __fadd_rn(p1, o1);
            }
        }
        S = __shfl_sync(FULL, v, 0);
        pen0 = __shfl_sync(FULL, p0, 0);
        pen1 = __shfl_sync(FULL, p1, 0);
    }

    // the k least reliable positions (|alpha|, ties to the lower index)
    __device__ void node_least(int lam, int k, int *m, float *mag) const {
        if (!PCK(lam >= 0 && lam <= n && k <= 4)) return;
        const int len = 1 << lam;
        const float *A = stage(lam);
        if (len > 32) {
            const Least r = node_least_wide(A, len, k, lane);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                m[j] = r.m[j];
                mag[j] = r.mag[j];
            }
            return;
        }
        {  // one value per lane: k rounds of warp minima
            uint32_t v = lane < len ? __float_as_uint(fabsf(A[lane])) : EMPTY;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (j >= k) break;
                const uint32_t gv = __reduce_min_sync(FULL, v);
                const uint32_t gi = __reduce_min_sync(FULL, v == gv ? uint32_t(lane) : EMPTY);
                m[j] = int(gi);
                mag[j] = __uint_as_float(gv);
                if (uint32_t(lane) == gi) v = EMPTY;
            }
        }
    }

    // flip the candidate's positions relative to the node's hard decisions
    __device__ void apply_flips(uint32_t mask, const int *m, int s, int lam) const {
#ifdef POLAR_DEBUG
        bool in = lam >= 0 && lam <= n && s >= 0 && s + (1 << lam) <= N();
        for (int j = 0; j < 4; ++j)
            if ((mask >> j) & 1u) in = in && m[j] >= 0 && m[j] < (1 << lam);
        if (!PCK(in)) {
            __syncwarp();
            return;
        }
#endif
        if (lam <= 5) {  // the node lies in one word: one masked XOR
            if (lane == 0 && mask) {
                uint32_t x = (mask & FLIP_ALL) ? ((lam == 5) ? FULL : ((1u << (1 << lam)) - 1u)) : 0u;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if ((mask >> j) & 1u) x ^= 1u << m[j];
                beta[s >> 5] ^= x << (s & 31);
            }
            __syncwarp();
            return;
        }
        if (mask & FLIP_ALL) {
            const int len = 1 << lam;
            if (len >= 32) {
                #pragma unroll 1
                for (int k = lane; k < (len >> 5); k += 32) beta[(s >> 5) + k] ^= FULL;
            } else if (lane == 0) {
                beta[s >> 5] ^= ((1u << len) - 1u) << (s & 31);
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if ((mask >> j) & 1u) {
                    const int pos = s + m[j];
                    beta[pos >> 5] ^= 1u << (pos & 31);
                }
        }
        __syncwarp();
    }
};

// The stack of one frame: entry j * 32 + lane lives in slot j of `lane`
// (NS = 1 holds D <= 32 entries, NS = 2 up to 64).
template <int NS>
struct Stack {
    uint32_t pm[NS], meta[NS], seq[NS], aux[NS];  // meta = len | sched << 16
};
template <>
struct Stack<0> {};  // the memory stack keeps nothing in registers

__device__ __forceinline__ bool slot_exists(int j, int lane, int D) { return j * 32 + lane < D; }

// Candidates of one expansion, described compactly so that every lane can
// produce any candidate r from registers: flip mask r is nibble r of `masks`
// (REP: candidate 1 flips all), and its path-metric delta is the ascending
// sum of the flipped positions' |alpha| (REP: rep0 / rep1).
struct Cands {
    int nc;
    uint32_t masks;
    bool rep;
    float rep0, rep1;
    float mag[4];

    __device__ __forceinline__ uint32_t mask(int r) const { return rep ? (r ? FLIP_ALL : 0u) : ((masks >> (4 * r)) & 0xFu); }
    __device__ __forceinline__ float delta(int r) const {
        if (rep) return r ? rep1 : rep0;
        const uint32_t mk = (masks >> (4 * r)) & 0xFu;
        float d = 0.0f;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if ((mk >> j) & 1u) d = __fadd_rn(d, mag[j]);
        return d;
    }
};

// CRC syndrome of the codeword estimate in beta: zero iff the message's CRC
// matches (the long division is linear, so the syndrome is a fixed GF(2)
// matrix applied to the codeword bits)
__device__ __noinline__ bool crc_ok(const Code &c, const uint32_t *beta, int lane) {
    uint32_t syn = 0u;
    for (int r = 0; r < c.crc; ++r) {
        uint32_t par = 0u;
        #pragma unroll 1
        for (int k = lane; k < c.W; k += 32) par ^= __popc(beta[k] & __ldg(c.crc_rows + size_t(r) * c.W + k));
        syn |= (par & 1u) << r;
    }
    return __reduce_xor_sync(FULL, syn) == 0u;
}

// output: re-encode the codeword estimate (F is an involution, Sec. 2.2.2)
// and read the message bits off the information set; a systematic code
// carries them in the codeword estimate itself
__device__ __noinline__ int write_output(const Code &c, uint32_t *u, uint32_t *orow, int lane) {
    int bad = 0;
    const int W = c.W, N = c.N;
    if (!c.systematic) {
        #pragma unroll 1
        for (int k = lane; k < W; k += 32) {
            uint32_t x = u[k];
            if (N > 1) x ^= (x >> 1) & 0x55555555u;
            if (N > 2) x ^= (x >> 2) & 0x33333333u;
            if (N > 4) x ^= (x >> 4) & 0x0F0F0F0Fu;
            if (N > 8) x ^= (x >> 8) & 0x00FF00FFu;
            if (N > 16) x ^= (x >> 16) & 0x0000FFFFu;
            u[k] = x;
        }
        __syncwarp();
        for (int hw = 1; hw < W; hw <<= 1) {
            #pragma unroll 1
            for (int k = lane; k < W; k += 32)
                if (!(k & hw)) u[k] ^= u[k + hw];
            __syncwarp();
        }
    }
    #pragma unroll 1
    for (int ow = lane; ow < c.info_words; ow += 32) {
        uint32_t word = 0u;
        for (int bb = 0; bb < 32; ++bb) {
            const int j = ow * 32 + bb;
            if (j < c.Kmsg) {
                const int p = __ldg(c.msg_pos + j);
                if (PCK(p >= 0 && p < c.N)) word |= ((u[p >> 5] >> (p & 31)) & 1u) << bb;
            }
        }
        orow[ow] = word;
    }
    __syncwarp();
    return bad;
}

// ---- stack and snapshot bookkeeping (plain inline functions: the stack
// stays in registers) ----

// insert candidates 0..nc-1 in order (reading R11): free slots first, all at
// once, then one by one, each replacing the worst entry (largest pm, ties:
// oldest) only if its pm is strictly smaller
template <int NS>
__device__ __forceinline__ void insert_cands(Stack<NS> &st, int &count, const Cands &c, float pm, uint32_t meta,
                                             uint32_t base, uint32_t slot, int D, int lane) {
    const int nfree = D - count;
    const int nb = c.nc < nfree ? c.nc : nfree;
    // lane r forms candidate r's metric once; the loops below read it
    const uint32_t my_pmb = __float_as_uint(__fadd_rn(pm, c.delta(lane < c.nc ? lane : 0)));
    if (nb > 0) {
        const uint32_t lt = (1u << lane) - 1u;
        int before = 0;  // free slots in the rows above
#pragma unroll
        for (int j = 0; j < NS; ++j) {
            const bool f = st.pm[j] == EMPTY && slot_exists(j, lane, D);
            const uint32_t bj = __ballot_sync(FULL, f);
            const int r = before + __popc(bj & lt);
            const uint32_t rpmb = __shfl_sync(FULL, my_pmb, r & 31);
            if (f && r < nb) {
                st.pm[j] = rpmb;
                st.meta[j] = meta;
                st.seq[j] = base + uint32_t(c.nc - 1 - r);
                st.aux[j] = slot | (c.mask(r) << 8);
            }
            before += __popc(bj);
        }
        count += nb;
    }
    // a full stack: only candidates below the current worst entry can enter,
    // and the worst only falls as they do, so the others are skipped at once;
    // the worst entry is found again only after a replacement
    uint32_t lw = 0u, ls = EMPTY, gw = 0u;
    int lj = 0;
    bool stale = true;
    uint32_t todo = 0u;  // candidates below the worst entry (it only decreases)
    if (nb < c.nc) {
        const bool e0 = slot_exists(0, lane, D);
        lw = e0 ? st.pm[0] : 0u;
        ls = e0 ? st.seq[0] : EMPTY;
#pragma unroll
        for (int j = 1; j < NS; ++j)
            if (slot_exists(j, lane, D) && (st.pm[j] > lw || (st.pm[j] == lw && st.seq[j] < ls))) {
                lw = st.pm[j];
                ls = st.seq[j];
                lj = j;
            }
        gw = __reduce_max_sync(FULL, lw);
        stale = false;
        todo = __ballot_sync(FULL, lane >= nb && lane < c.nc && my_pmb < gw);
    }
    while (todo) {
        const int k = __ffs(todo) - 1;
        todo &= todo - 1u;
        const uint32_t pmb = __shfl_sync(FULL, my_pmb, k);
        if (stale) {
            const bool e0 = slot_exists(0, lane, D);
            lw = e0 ? st.pm[0] : 0u;
            ls = e0 ? st.seq[0] : EMPTY;
            lj = 0;
#pragma unroll
            for (int j = 1; j < NS; ++j)
                if (slot_exists(j, lane, D) && (st.pm[j] > lw || (st.pm[j] == lw && st.seq[j] < ls))) {
                    lw = st.pm[j];
                    ls = st.seq[j];
                    lj = j;
                }
            gw = __reduce_max_sync(FULL, lw);
            stale = false;
        }
        if (pmb < gw) {
            stale = true;
            const uint32_t gs = __reduce_min_sync(FULL, lw == gw ? ls : EMPTY);
            const uint32_t bal = __ballot_sync(FULL, lw == gw && ls == gs);
            if (lane == __ffs(bal) - 1) {
#pragma unroll
                for (int j = 0; j < NS; ++j)
                    if (lj == j) {
                        st.pm[j] = pmb;
                        st.meta[j] = meta;
                        st.seq[j] = base + uint32_t(c.nc - 1 - k);
                        st.aux[j] = slot | (c.mask(k) << 8);
                    }
            }
        }
    }
}

// a free snapshot slot among 0 .. D-1 (one always exists: the extended path
// left the stack, so at most D - 1 snapshots are referenced)
template <int NS>
__device__ __forceinline__ int alloc_snapshot(const Stack<NS> &st, int D) {
    if constexpr (NS == 1) {  // D <= 32: slot ids below 32, one word
        uint32_t used = 0u;
        const uint32_t sn = st.aux[0] & 0xFFu;
        if (st.pm[0] != EMPTY && sn < 32u) used = 1u << sn;
        used = __reduce_or_sync(FULL, used);
        const uint32_t fr = ~used & (D >= 32 ? FULL : ((1u << D) - 1u));
        return fr ? (__ffs(int(fr)) - 1) : -1;
    }
    uint32_t lo = 0u, hi = 0u;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
        if (st.pm[j] != EMPTY) {
            const uint32_t sn = st.aux[j] & 0xFFu;
            if (sn < 32u) lo |= 1u << sn;
            else if (sn < 64u) hi |= 1u << (sn - 32u);
        }
    }
    lo = __reduce_or_sync(FULL, lo);
    hi = __reduce_or_sync(FULL, hi);
    const uint64_t used = (uint64_t(hi) << 32) | uint64_t(lo);
    const uint64_t all = (D >= 64) ? ~0ull : ((1ull << D) - 1ull);
    const uint64_t fr = ~used & all;
    return fr ? (__ffsll((long long)fr) - 1) : -1;
}

__device__ __forceinline__ void write_snapshot(const Warp &w, int W, int SW, int slot, int nbits, uint32_t m01,
                                               uint32_t m23, int s, int lam) {
    uint32_t *sp = w.scr + size_t(slot) * SW;
    const int nw = min(W, (nbits + 31) >> 5);
    #pragma unroll 1
    for (int k = w.lane; k < nw; k += 32) sp[k] = w.beta[k];
    if (w.lane == 0) {
        sp[W] = m01;
        sp[W + 1] = m23;
        sp[W + 2] = uint32_t(s);
        sp[W + 3] = uint32_t(lam);
    }
    __syncwarp();
}

// ---- the memory stack (depths above 64, e.g. the D = 8192 of Sec. 5) ----
// Entries {pm bits, meta, seq, aux} are dense in [0, count) of a per-warp
// region of global scratch (aux = snapshot slot | flip mask << 24); for each
// block of 32 entries shared memory holds {pm bits, seq} of its best entry
// (smallest pm, ties newest), so a pop reads the block bests, then one block.
// A popped entry's hole is filled by the last entry.  The order rules are
// those of the register stack.
struct MemStack {
    uint4 *e;     // global: the entries
    uint2 *best;  // shared: best entry per block of 32
    int cap;      // entries the region holds
};

struct Popped {
    uint32_t pmb, meta, aux;
    int ok;
};

struct Worst {
    uint32_t pm;
    int idx;
};

// best[blk] from the block's entries below `count`
__device__ __noinline__ void mem_block_best(MemStack ms, int blk, int count, int lane) {
    const int i = blk * 32 + lane;
    const uint4 v = i < count ? ms.e[i] : make_uint4(EMPTY, 0u, 0u, 0u);
    const uint32_t gp = __reduce_min_sync(FULL, v.x);
    const uint32_t gs = __reduce_max_sync(FULL, v.x == gp ? v.z : 0u);
    if (lane == 0) ms.best[blk] = make_uint2(gp, gs);
    __syncwarp();
}

// remove and return the best entry (smallest pm, ties newest); ok = 0 if
// there is none or the block bests disagree with the entries
__device__ __noinline__ Popped mem_pop(MemStack ms, int count, int lane) {
    Popped r{EMPTY, 0u, 0u, 0};
    const int nb = (count + 31) >> 5;
    uint32_t bp = EMPTY, bs = 0u;
    int bb = 0;
    #pragma unroll 1
    for (int k = lane; k < nb; k += 32) {
        const uint2 v = ms.best[k];
        if (v.x < bp || (v.x == bp && v.y > bs)) {
            bp = v.x;
            bs = v.y;
            bb = k;
        }
    }
    const uint32_t gp = __reduce_min_sync(FULL, bp);
    if (gp == EMPTY) return r;
    const uint32_t gs = __reduce_max_sync(FULL, bp == gp ? bs : 0u);
    const uint32_t bal = __ballot_sync(FULL, bp == gp && bs == gs);
    const int blk = __shfl_sync(FULL, bb, __ffs(bal) - 1);
    const int i = blk * 32 + lane;
    const uint4 v = i < count ? ms.e[i] : make_uint4(EMPTY, 0u, 0u, 0u);
    const uint32_t hit = __ballot_sync(FULL, i < count && v.x == gp && v.z == gs);
    if (!hit) return r;
    const int wl = __ffs(hit) - 1;
    r.pmb = gp;
    r.meta = __shfl_sync(FULL, v.y, wl);
    r.aux = __shfl_sync(FULL, v.w, wl);
    const int hole = blk * 32 + wl, last = count - 1;
    if (hole != last && lane == 0) ms.e[hole] = ms.e[last];
    __syncwarp();
    mem_block_best(ms, blk, last, lane);
    const int lb = last >> 5;
    if (lb != blk && lb * 32 < last) mem_block_best(ms, lb, last, lane);
    r.ok = 1;
    return r;
}

// the worst of `count` >= 1 entries: largest pm, ties oldest
__device__ __noinline__ Worst mem_worst(MemStack ms, int count, int lane) {
    uint32_t lw = 0u, ls = EMPTY;
    int li = -1;
    #pragma unroll 1
    for (int i = lane; i < count; i += 32) {
        const uint4 v = ms.e[i];
        if (li < 0 || v.x > lw || (v.x == lw && v.z < ls)) {
            lw = v.x;
            ls = v.z;
            li = i;
        }
    }
    const uint32_t gw = __reduce_max_sync(FULL, li >= 0 ? lw : 0u);
    const uint32_t gs = __reduce_min_sync(FULL, (li >= 0 && lw == gw) ? ls : EMPTY);
    const uint32_t bal = __ballot_sync(FULL, li >= 0 && lw == gw && ls == gs);
    Worst w;
    w.pm = gw;
    w.idx = __shfl_sync(FULL, li, __ffs(bal) - 1);
    return w;
}

// insert candidates 0..nc-1 in order, as insert_cands does; returns the new
// count, or -1 if the region would overflow (cannot happen with the host's
// sizing: at most 1 + 7 entries per iteration)
__device__ __noinline__ int mem_insert(MemStack ms, int count, const Cands c, float pm, uint32_t meta, uint32_t base,
                                       uint32_t slot, int D, int lane) {
    const uint32_t my_pmb = __float_as_uint(__fadd_rn(pm, c.delta(lane < c.nc ? lane : 0)));
    const int nfree = D - count;
    const int nb = c.nc < nfree ? c.nc : nfree;
    if (count + nb > ms.cap) return -1;
    if (nb > 0) {
        if (lane < nb)
            ms.e[count + lane] = make_uint4(my_pmb, meta, base + uint32_t(c.nc - 1 - lane), slot | (c.mask(lane) << 24));
        __syncwarp();
        const int b0 = count >> 5, b1 = (count + nb - 1) >> 5;
        count += nb;
        mem_block_best(ms, b0, count, lane);
        if (b1 != b0) mem_block_best(ms, b1, count, lane);
    }
    if (nb < c.nc) {  // a full stack: strict replacement of the worst entry
        Worst w = mem_worst(ms, count, lane);
        uint32_t todo = __ballot_sync(FULL, lane >= nb && lane < c.nc && my_pmb < w.pm);
        bool stale = false;
        while (todo) {
            const int k = __ffs(todo) - 1;
            todo &= todo - 1u;
            const uint32_t pmb = __shfl_sync(FULL, my_pmb, k);
            if (stale) {
                w = mem_worst(ms, count, lane);
                stale = false;
            }
            if (pmb < w.pm) {
                if (lane == 0)
                    ms.e[w.idx] = make_uint4(pmb, meta, base + uint32_t(c.nc - 1 - k), slot | (c.mask(k) << 24));
                __syncwarp();
                mem_block_best(ms, w.idx >> 5, count, lane);
                stale = true;
            }
        }
    }
    return count;
}

// the L-prune: drop every entry of length <= s (order kept), rebuild the
// block bests; returns the new count
__device__ __noinline__ int mem_prune(MemStack ms, int count, int s, int lane) {
    const uint32_t lt = (1u << lane) - 1u;
    int out = 0;
    #pragma unroll 1
    for (int b0 = 0; b0 < count; b0 += 32) {
        const int i = b0 + lane;
        const uint4 v = i < count ? ms.e[i] : make_uint4(EMPTY, 0u, 0u, 0u);
        const bool keep = i < count && int(v.y & 0xFFFFu) > s;
        const uint32_t bal = __ballot_sync(FULL, keep);
        __syncwarp();  // the block is read before any lane writes into it
        if (keep) ms.e[out + __popc(bal & lt)] = v;
        out += __popc(bal);
    }
    __syncwarp();
    #pragma unroll 1
    for (int blk = 0; blk * 32 < out; ++blk) mem_block_best(ms, blk, out, lane);
    return out;
}

// NS = 1, 2: the register stack (D <= 32, 64); NS = 0: the memory stack `ms`
template <int NS, bool EXACT, bool STATS>
__device__ __forceinline__ void decode_frame(const Args &a, const Code &c, const int D, const int L, Warp &w,
                                             unsigned b, uint32_t *orow, const MemStack ms) {
    constexpr bool DEEP = NS == 0;
    constexpr bool CG = !DEEP;  // LLR and snapshot loads through L2 only
    constexpr uint32_t nosnap = DEEP ? NOSNAP_DEEP : NOSNAP;
    constexpr int mask_shift = DEEP ? 24 : 8;
    const int lane = w.lane;
#ifdef POLAR_DEBUG
    int &bad = w.bad;  // the index checks of this function mark the frame
#endif
    const int N = c.N, W = c.W, n = c.n;
    const int SW = c.snap_words;
    const int max_iter = L * (c.nbranch + 9) + 2;
    // snapshot slots: 0 .. D-1 reused (register stack) or one per iteration
    // (memory stack); the slot after them keeps the first complete path
    const int first_slot = DEEP ? max_iter : D;
    const uint32_t stack_cost = 2u * uint32_t(D > 2 ? 32 - __clz(D - 1) : 1);

    PT_INIT
    #pragma unroll 1
    for (int i = lane; i < c.nbranch; i += 32) w.cnt[i] = 0;
    #pragma unroll 1
    for (int i = lane; i < W; i += 32) w.beta[i] = 0u;
    __syncwarp();

    Stack<NS> st;
    if constexpr (DEEP) {
        if (lane == 0) {  // the initial path: pm 0, length 0, schedule 0
            ms.e[0] = make_uint4(__float_as_uint(0.0f), 0u, 0u, NOSNAP_DEEP);
            ms.best[0] = make_uint2(__float_as_uint(0.0f), 0u);
        }
        __syncwarp();
    } else {
#pragma unroll
        for (int j = 0; j < NS; ++j) {
            st.pm[j] = EMPTY;
            st.meta[j] = 0u;
            st.seq[j] = 0u;
            st.aux[j] = NOSNAP;
        }
        if (lane == 0) {  // the initial path: pm 0, length 0, schedule 0
            st.pm[0] = __float_as_uint(0.0f);
            st.meta[0] = 0u;
            st.seq[0] = 0u;
            st.aux[0] = NOSNAP;
        }
    }
    int count = 1;
    uint32_t seq_next = 1;
    uint32_t ops = stack_cost;  // counted operations (roofline convention)
    uint32_t n_iter = 0, n_switch = 0, n_exp = 0;

    uint32_t cur_snap = nosnap;  // snapshot of the latest expansion
    bool beta_dirty = false;     // working beta replaced since that expansion
    uint32_t applied = 0;        // flips applied on top of the latest snapshot
    int cm[4] = {0, 0, 0, 0};
    int cs = 0, clam = n;        // node of the latest expansion
    // alpha stages valid_lo .. n-1 hold the spine of node (clam, cs),
    // computed from the working beta's prefix (n: none valid)
    int cur_lo = n, valid_lo = n;

    int crc_fails = 0;
    bool have_first = false;
    float first_pm = 0.0f;
    int status = POLAR_TIMEOUT;
    float out_pm = __int_as_float(0x7f800000);
    int out_src = 0;  // 0: zeros, 1: working beta, 2: first complete path

    int iter = 0;
    for (; iter < max_iter; ++iter) {
        if (count == 0) {  // every path deleted (reading R12)
            status = POLAR_CRC_FAIL;
            if (have_first) {
                out_pm = first_pm;
                out_src = 2;
            }
            break;
        }
        // ---- pop the best path: smallest pm, ties to the newest ----
        uint32_t p_pmb, p_meta, p_aux;
        if constexpr (DEEP) {
            const Popped pp = mem_pop(ms, count, lane);
            if (!pp.ok) {  // count out of step with the entries: stop safely
                status = POLAR_TIMEOUT;
                break;
            }
            p_pmb = pp.pmb;
            p_meta = pp.meta;
            p_aux = pp.aux;
        } else {
            uint32_t lp = st.pm[0], ls = st.seq[0];
            int lj = 0;
#pragma unroll
            for (int j = 1; j < NS; ++j)
                if (st.pm[j] < lp || (st.pm[j] == lp && st.pm[j] != EMPTY && st.seq[j] > ls)) {
                    lp = st.pm[j];
                    ls = st.seq[j];
                    lj = j;
                }
            const uint32_t gp = __reduce_min_sync(FULL, lp);
            if (gp == EMPTY) {  // count out of step with the slots: stop safely
                status = POLAR_TIMEOUT;
                break;
            }
            const uint32_t gs = __reduce_max_sync(FULL, lp == gp ? ls : 0u);
            const uint32_t bal = __ballot_sync(FULL, lp == gp && ls == gs);
            const int wl = __ffs(bal) - 1;
            p_pmb = gp;
            uint32_t my_meta = st.meta[0], my_aux = st.aux[0];  // this lane's best entry
#pragma unroll
            for (int j = 1; j < NS; ++j)
                if (lj == j) {
                    my_meta = st.meta[j];
                    my_aux = st.aux[j];
                }
            p_meta = __shfl_sync(FULL, my_meta, wl);
            p_aux = __shfl_sync(FULL, my_aux, wl);
            if (lane == wl) {
#pragma unroll
                for (int j = 0; j < NS; ++j)
                    if (lj == j) st.pm[j] = EMPTY;
            }
        }
        --count;
        ++n_iter;
        ops += stack_cost;
        const int p_sched = int(p_meta >> 16);
        const uint32_t p_snap = p_aux & nosnap;
        const uint32_t p_mask = (p_aux >> mask_shift) & 0x1Fu;
        if (p_snap != nosnap && p_snap >= uint32_t(first_slot)) {  // never produced; guards the scratch index
            status = POLAR_TIMEOUT;
            break;
        }
        if (p_sched > c.nops) {
            status = POLAR_TIMEOUT;
            break;
        }
        PT(PH_POP)

        // ---- restore the path's beta array ----
        bool switched = false;
        int div = 0;  // first bit where the popped path's beta differs from the working one
        if (p_snap == cur_snap) {
            if (beta_dirty) {
                const uint32_t *sp = w.scr + size_t(cur_snap) * SW;
                #pragma unroll 1
                for (int k = lane; k < W; k += 32) w.beta[k] = ld_l2<CG>(sp + k);
                __syncwarp();
                applied = 0u;
                beta_dirty = false;
                valid_lo = cur_lo;
            }
            if (applied ^ p_mask) w.apply_flips(applied ^ p_mask, cm, cs, clam);
            applied = p_mask;
        } else {  // path switch (Sec. 3.3)
#ifdef POLAR_DEBUG
            {  // the snapshot's node must lie inside the code
                const uint32_t *sp = w.scr + size_t(p_snap) * SW;
                const int ss = int(sp[W + 2]), slam = int(sp[W + 3]);
                if (!w.PCK_snap(ss, slam)) {
                    status = POLAR_TIMEOUT;
                    break;
                }
            }
#endif
            switched = true;
            ++n_switch;
            ops += uint32_t(W);
            div = (CG ? restore_switch_cg : restore_switch)(w.scr + size_t(p_snap) * SW, w.beta, W, p_mask, lane);
            beta_dirty = true;
        }
        PT(PH_BETA)

        if (p_sched == c.nops) {  // a complete path
            if (switched) valid_lo = n;  // beta replaced, alpha left as it was
            bool pass = true;
            if (c.crc) {
                ops += uint32_t(c.crc) * uint32_t(W);
                pass = crc_ok(c, w.beta, lane);
            }
            if (pass) {
                status = POLAR_OK;
                out_pm = __uint_as_float(p_pmb);
                out_src = 1;
                break;
            }
            ++crc_fails;
            if (!have_first) {
                have_first = true;
                first_pm = __uint_as_float(p_pmb);
                uint32_t *sp = w.scr + size_t(first_slot) * SW;
                #pragma unroll 1
                for (int k = lane; k < W; k += 32) sp[k] = w.beta[k];
                __syncwarp();
            }
            if (crc_fails >= L) {
                status = POLAR_CRC_FAIL;
                out_pm = first_pm;
                out_src = 2;
                break;
            }
            PT(PH_DONE)
            continue;
        }

        // ---- alpha after a switch (Alg. calp): recompute the spine from the
        // channel, except the top stages the popped path shares with the
        // spine held now (same node, identical beta before the node).  The
        // recomputed stages rl .. lam_d run through the same op dispatch as
        // the schedule walk below. ----
        int rl = -1, lam_d = 0, s_d = 0;
        if (switched) {
            const uint32_t tgt = __ldg(&c.ops[p_sched].z);
            if (tgt != NO_TARGET) {
                lam_d = int(tgt & 0xFFu);
                s_d = int(tgt >> 8);
                ops += 2u * uint32_t(N - (1 << lam_d));  // counted as the full recompute
                // each condition of the reuse test holds on a range lam >= T_k,
                // so the first stage to recompute is one below their maximum
                const uint32_t xs = uint32_t(s_d ^ cs);
                int T = max(lam_d, valid_lo);
                if (xs) T = max(T, 32 - __clz(xs));
                if (div < s_d) T = max(T, 32 - __clz(uint32_t(s_d ^ div)));
                rl = min(n - 1, T - 1);
            }
        }
        PT(PH_ALPHA)

        // ---- walk the schedule to the next branching node (Sec. 4) ----
        float pm = __uint_as_float(p_pmb);
        int t = p_sched;
        const uint4 *opsv = reinterpret_cast<const uint4 *>(c.ops);
        uint4 nxt = __ldg(opsv + min(t, c.nops - 1));
        uint4 op = nxt;
        for (;;) {
            uint32_t code;
            int lam, s, run = 1;
            const bool sched = rl < lam_d;  // else: a recomputed spine stage
            if (!sched) {
                lam = rl;
                s = (s_d >> lam) << lam;
                code = ((s_d >> lam) & 1) ? OP_G : OP_F;
                --rl;
            } else {
                if (t >= c.nops) break;
                op = nxt;
                if (t + 1 < c.nops) nxt = __ldg(opsv + t + 1);
                code = op.x & 0xFFu;
                lam = int((op.x >> 8) & 0xFFu);
                s = int(op.y);
                run = int((op.x >> 16) & 0xFFu) + 1;
                if (code >= OP_BRANCH) break;
                ++t;
            }
            if (code <= OP_G) {  // an F or G, then run - 1 F ops down the left edge
                #pragma unroll 1
                for (int i = 0; i < run; ++i) {
                    if (i == 0 && code == OP_G) w.template op_g<CG>(lam, s);
                    else w.template op_f<EXACT, CG>(lam - i);
                    if (sched) ops += 2u << (lam - i);
                }
                PT(PH_FG)
            } else if (code == OP_COMB) {  // run combines, one stage up each
                #pragma unroll 1
                for (int i = 0; i < run; ++i) {
                    w.op_comb(lam + i, s);
                    ops += (lam + i < 5) ? 1u : (1u << (lam + i - 5));
                    s -= 1 << (lam + i);
                }
                PT(PH_COMB)
            } else {  // Rate-0 node or frozen leaf: beta = 0, PM += sum HD(a)|a|
                const float pen = w.node_sum(lam, EXACT ? 3 : 1);
                w.set_range(lam, s, 0u);
                pm = __fadd_rn(pm, pen);
                ops += (2u << lam) + 1u;
                PT(PH_R0)
            }
        }
        ++n_exp;

        // ---- the expansion's candidates: a complete path is pushed as it
        // is; a branching node gets its visit counter, the L-prune
        // (Sec. 2.2.5) and the node candidates (Sec. 2.2.4, readings R7-R9) ----
        Cands cd{0, 0u, false, 0.0f, 0.0f, {0.0f, 0.0f, 0.0f, 0.0f}};
        int m[4] = {0, 0, 0, 0};
        int node_s = 0, node_lam = n, snap_lam = 0, nbits = N;
        uint32_t meta = uint32_t(N) | (uint32_t(c.nops) << 16);
        if (t >= c.nops) {
            cd.nc = 1;
            ops += 1u;
        } else {
            const uint32_t code = op.x & 0xFFu;
            const int lam = int((op.x >> 8) & 0xFFu);
            const int s = int(op.y);
            const int len = 1 << lam;
            node_s = s;
            node_lam = snap_lam = lam;
            nbits = s + len;
            meta = uint32_t(s + len) | (uint32_t(t + 1) << 16);
            uint32_t vc = 0;
            if (lane == 0 && PCK(int(op.w) < c.nbranch)) vc = ++w.cnt[op.w];
            vc = __shfl_sync(FULL, vc, 0);
            __syncwarp();
            if (int(vc) >= L) {
                ops += stack_cost;
                if constexpr (DEEP) {
                    count = mem_prune(ms, count, s, lane);
                } else {
                    int removed = 0;
#pragma unroll
                    for (int j = 0; j < NS; ++j) {
                        const bool kill = st.pm[j] != EMPTY && int(st.meta[j] & 0xFFFFu) <= s;
                        removed += __popc(__ballot_sync(FULL, kill));
                        if (kill) st.pm[j] = EMPTY;
                    }
                    count -= removed;
                }
            }
            PT(PH_PRUNE)

            if (code == OP_REP) {
                float S, p0;
                uint32_t bbit;
                if (len <= 32) {
                    float pz, po;
                    w.rep_sums(lam, S, pz, po);
                    bbit = S < 0.0f ? 1u : 0u;
                    p0 = bbit ? po : pz;
                } else {
                    S = w.node_sum(lam, 0);
                    bbit = S < 0.0f ? 1u : 0u;
                    p0 = w.node_sum(lam, bbit ? 2 : 1);
                }
                w.set_range(lam, s, bbit);
                cd.nc = 2;
                cd.rep = true;
                cd.rep0 = p0;
                cd.rep1 = __fadd_rn(p0, fabsf(S));
                ops += 4u * uint32_t(len) + 3u;
            } else {  // information leaf, Rate-1 or SPC: hard decisions first
                const uint32_t q = w.node_hd(lam, s);
                if (code == OP_LEAF1 && EXACT) {  // ln(1 + e^-|a|), ln(1 + e^|a|)
                    const float aa = fabsf(w.stage(0)[0]);
                    cd.nc = 2;
                    cd.rep = true;
                    cd.rep0 = softplus_f(-aa);
                    cd.rep1 = softplus_f(aa);
                    ops += 4u;
                } else if (code == OP_LEAF1) {
                    cd.mag[0] = fabsf(w.stage(0)[0]);
                    cd.nc = 2;
                    cd.masks = LEAF1_MASKS;
                    ops += 4u;
                } else {
                    const bool spc = code == OP_SPC;
                    w.node_least(lam, spc ? 4 : 2, m, cd.mag);
                    cd.nc = spc ? 8 : 4;
                    cd.masks = spc ? (q ? SPC_MASKS_ODD : SPC_MASKS_EVEN) : R1_MASKS;
                    ops += spc ? 10u * uint32_t(len) + (q ? 16u : 17u) : 6u * uint32_t(len) + 5u;
                }
            }
            PT(PH_NODE)
        }

        int slot;
        if constexpr (DEEP) slot = iter;  // one slot per iteration, never reused
        else slot = alloc_snapshot(st, D);
        if (slot < 0) break;
        write_snapshot(w, W, SW, slot, nbits, uint32_t(m[0]) | (uint32_t(m[1]) << 16),
                       uint32_t(m[2]) | (uint32_t(m[3]) << 16), node_s, snap_lam);
        cur_snap = uint32_t(slot);
        applied = 0u;
        beta_dirty = false;
        cm[0] = m[0];
        cm[1] = m[1];
        cm[2] = m[2];
        cm[3] = m[3];
        cs = node_s;
        clam = node_lam;
        cur_lo = valid_lo = node_lam;
        PT(PH_SNAP)
        ops += uint32_t(cd.nc) * stack_cost;
        if constexpr (DEEP) {
            count = mem_insert(ms, count, cd, pm, meta, seq_next, uint32_t(slot), D, lane);
            if (count < 0) {  // the entry region is full (excluded by its sizing)
                status = POLAR_TIMEOUT;
                break;
            }
        } else {
            insert_cands(st, count, cd, pm, meta, seq_next, uint32_t(slot), D, lane);
        }
        seq_next += uint32_t(cd.nc);
        PT(PH_INSERT)
    }

    // ---- output ----
    if (out_src == 2) {
        const uint32_t *sp = w.scr + size_t(first_slot) * SW;
        #pragma unroll 1
        for (int k = lane; k < W; k += 32) w.beta[k] = ld_l2<CG>(sp + k);
    } else if (out_src == 0) {
        #pragma unroll 1
        for (int k = lane; k < W; k += 32) w.beta[k] = 0u;
    }
    __syncwarp();
    if (!c.systematic) ops += uint32_t(n) * uint32_t(W);
    const int out_bad = write_output(c, w.beta, orow, lane);
#ifdef POLAR_DEBUG
    if (__any_sync(FULL, w.bad || out_bad)) status = POLAR_DEBUG_FAIL;
#else
    (void)out_bad;
#endif
    if (lane == 0) {
        if (status == POLAR_TIMEOUT || status == POLAR_DEBUG_FAIL) out_pm = __int_as_float(0x7f800000);
        a.pm_out[b] = out_pm;
        a.status_out[b] = int8_t(status);
        if (STATS && a.stats_out) {  // without counters all counting is dead code
            uint32_t *sr = a.stats_out + size_t(b) * 4;
            sr[0] = n_iter;
            sr[1] = n_switch;
            sr[2] = ops;
            sr[3] = n_exp;
        }
    }
    __syncwarp();
    PT(PH_OUT)
    PT_FLUSH
}

// One warp per frame, persistent: warps claim `chunk` frames at a time.
// MIXED = false: every frame uses a.code, a.D, a.L and row b of the LLR and
// message buffers.  MIXED = true: frame b has its own code, D and L
// (a.frames[b]) and offsets into packed LLR and message buffers.
// Blocks per SM (registers per thread): measured per instantiation.  The
// one-row min-sum decoder runs fastest at 9 (56 registers; 8: 1.3 % slower,
// 7: 6 %, 10: 19 %); the memory stack at 8 (9: 11 % slower, 7: 7 %); the mixed
// decoders at 6, which their shared memory allows for codes up to N = 2048.
template <bool MIXED, int NS, bool EXACT>
constexpr int decode_blocks_per_sm() { return MIXED ? 6 : ((NS == 1 && !EXACT) ? 9 : 8); }

template <bool MIXED, int NS, bool EXACT, bool STATS>
__global__ void __launch_bounds__(128, decode_blocks_per_sm<MIXED, NS, EXACT>()) scs_decode_kernel(Args a) {
    extern __shared__ __align__(16) unsigned char smem[];
    Code *codes_s = reinterpret_cast<Code *>(smem);  // mixed: the set's codes (a.codes_smem bytes)
    if (MIXED) {
        for (int i = threadIdx.x; i < a.ncodes; i += blockDim.x) codes_s[i] = a.codes[i];
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned char *my = smem + a.codes_smem + size_t(wib) * a.warp_smem;
    const int gwarp = blockIdx.x * (blockDim.x >> 5) + wib;
    uint32_t *scr = a.scratch + size_t(gwarp) * size_t(a.scratch_stride);
    for (;;) {
        unsigned b0 = 0;
        if (lane == 0) b0 = atomicAdd(a.counter, unsigned(a.chunk));
        b0 = __shfl_sync(FULL, b0, 0);
        if (b0 >= unsigned(a.B)) break;
        const unsigned b1 = min(unsigned(a.B), b0 + unsigned(a.chunk));
        for (unsigned k = b0; k < b1; ++k) {
            const unsigned b = (MIXED && a.order) ? unsigned(__ldg(a.order + k)) : k;
            if (MIXED && b >= unsigned(a.nframes)) continue;
            if constexpr (!MIXED) {
                const Code &c = a.code;
                Warp w{lane, c.n, a.llr_vec, reinterpret_cast<float *>(my), reinterpret_cast<uint32_t *>(my + 4 * c.N),
                       my + 4 * c.N + 4 * c.W, scr, a.llr + size_t(b) * c.N, c.scales, 0};
                MemStack ms{nullptr, nullptr, 0};
                if constexpr (NS == 0)
                    ms = MemStack{reinterpret_cast<uint4 *>(scr + a.deep_ent_off),
                                  reinterpret_cast<uint2 *>(my + a.deep_best_off), a.deep_cap};
                decode_frame<NS, EXACT, STATS>(a, c, a.D, a.L, w, b, a.info_out + size_t(b) * c.info_words, ms);
            } else {
                const int4 fd = a.frames[b];
                if (fd.x < 0 || fd.x >= a.ncodes || fd.y < 1 || fd.y > a.Dmax || fd.z < 1 || fd.z > 255) {
                    if (lane == 0) {  // invalid descriptor: nothing is read or written but the status
                        a.pm_out[b] = __int_as_float(0x7f800000);
                        a.status_out[b] = int8_t(kBadFrame);
                    }
                    continue;
                }
                const Code &c = codes_s[fd.x];
                const long long lo = a.llr_off[b];
                Warp w{lane, c.n, (a.llr_vec && (lo & 3) == 0) ? 1 : 0, reinterpret_cast<float *>(my),
                       reinterpret_cast<uint32_t *>(my + 4 * c.N), my + 4 * c.N + 4 * c.W, scr, a.llr + lo, c.scales, 0};
                decode_frame<NS, false, STATS>(a, c, fd.y, fd.z, w, b, a.info_out + a.info_off[b], MemStack{nullptr, nullptr, 0});
            }
        }
    }
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Served requests (continuous batching): warps claim request indices in
// order, wait until the host has published the request (its LLRs copied into
// the arena), decode it as a mixed-batch frame, stamp the completion time and
// raise its completion flag in host-mapped memory.  Every wait is bounded:
// after wait_ns (or when the host raises abort_flag) the warp records an
// error and leaves.  Request LLRs live in an arena the host refills once the
// requests that used it have completed; since an SM's L1 may still hold lines
// of an earlier request there, a warp first copies its request's LLRs with
// L2-only loads into its own staging area (its own stores keep its L1
// coherent) and decodes from that copy.
template <int NS>
__global__ void __launch_bounds__(128, 6) scs_serve_kernel(Args a) {
    extern __shared__ __align__(16) unsigned char smem[];
    Code *codes_s = reinterpret_cast<Code *>(smem);  // the set's codes (a.codes_smem bytes)
    for (int i = threadIdx.x; i < a.ncodes; i += blockDim.x) codes_s[i] = a.codes[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned char *my = smem + a.codes_smem + size_t(wib) * a.warp_smem;
    const int gwarp = blockIdx.x * (blockDim.x >> 5) + wib;
    uint32_t *scr = a.scratch + size_t(gwarp) * size_t(a.scratch_stride);
    for (;;) {
        unsigned k = 0;
        int ok = 1;
        if (lane == 0) {
            k = atomicAdd(a.counter, 1u);
            if (k < unsigned(a.B)) {
                const unsigned long long t0 = global_ns();
                unsigned ns = 64;
                while (*reinterpret_cast<const volatile unsigned long long *>(a.head) <= k) {
                    if (*reinterpret_cast<const volatile int *>(a.abort_flag) || global_ns() - t0 > a.wait_ns) {
                        ok = 0;
                        atomicExch(a.error_flag, 1);
                        break;
                    }
                    __nanosleep(ns);
                    if (ns < 8192) ns <<= 1;
                }
                __threadfence();
            }
        }
        k = __shfl_sync(FULL, k, 0);
        ok = __shfl_sync(FULL, ok, 0);
        if (k >= unsigned(a.B) || !ok) break;
        if (lane == 0) a.t_start[k] = global_ns();
        const int4 fd = a.frames[k];
        if (fd.x < 0 || fd.x >= a.ncodes || fd.y < 1 || fd.y > a.Dmax || fd.z < 1 || fd.z > 255) {
            if (lane == 0) {
                a.pm_out[k] = __int_as_float(0x7f800000);
                a.status_out[k] = int8_t(kBadFrame);
            }
        } else {
            const Code &c = codes_s[fd.x];
            const float *src = a.llr + a.llr_off[k];
            float *stage = reinterpret_cast<float *>(scr + a.serve_stage_off);
            #pragma unroll 1
            for (int i = lane; i < c.N; i += 32) stage[i] = __ldcg(src + i);
            __syncwarp();
            Warp w{lane, c.n, 1, reinterpret_cast<float *>(my), reinterpret_cast<uint32_t *>(my + 4 * c.N),
                   my + 4 * c.N + 4 * c.W, scr, stage, c.scales, 0};
            decode_frame<NS, false, false>(a, c, fd.y, fd.z, w, k, a.info_out + a.info_off[k], MemStack{nullptr, nullptr, 0});
        }
        if (lane == 0) {
            a.t_done[k] = global_ns();
            __threadfence_system();
            reinterpret_cast<volatile unsigned char *>(a.done_flag)[k] = 1;
        }
        __syncwarp();
    }
}

__global__ void read_global_ns(unsigned long long *out) { *out = global_ns(); }

}  // namespace

Code make_code(const polar_plan *p, const KOp *ops, const uint32_t *crc_rows, const uint16_t *msg_pos,
               const float *scales) {
    Code c{};
    c.ops = ops;
    c.scales = p->scales.empty() ? nullptr : scales;
    c.crc_rows = crc_rows;
    c.msg_pos = msg_pos;
    c.N = p->N;
    c.n = p->n;
    c.W = p->W;
    c.Kmsg = p->Kmsg;
    c.crc = p->crc;
    c.nops = int(p->dev_ops.size());
    c.nbranch = p->nbranch;
    c.info_words = (p->Kmsg + 31) / 32;
    c.snap_words = ((p->W + 4) + 7) & ~7;
    c.systematic = p->systematic;
    return c;
}

int warp_smem_bytes(int N, int W, int nbranch) { return ((4 * N + 4 * W + nbranch) + 15) & ~15; }

// The instantiation of the decoder for one launch: mixed or uniform, one or
// two stack rows per lane, exact-f or min-sum, with or without counters.
template <bool MIXED, int NS, bool EXACT, bool STATS>
const void *kernel_fn() {
    return reinterpret_cast<const void *>(scs_decode_kernel<MIXED, NS, EXACT, STATS>);
}

const void *uniform_kernel(const polar_plan *p, int D, bool stats) {
    if (D > POLAR_MAX_D_GPU) return stats ? kernel_fn<false, 0, false, true>() : kernel_fn<false, 0, false, false>();
    const bool two = D > 32;
    if (p->exact) {
        if (two) return stats ? kernel_fn<false, 2, true, true>() : kernel_fn<false, 2, true, false>();
        return stats ? kernel_fn<false, 1, true, true>() : kernel_fn<false, 1, true, false>();
    }
    if (two) return stats ? kernel_fn<false, 2, false, true>() : kernel_fn<false, 2, false, false>();
    return stats ? kernel_fn<false, 1, false, true>() : kernel_fn<false, 1, false, false>();
}

const void *mixed_kernel(int Dmax, bool stats) {
    if (Dmax > 32) return stats ? kernel_fn<true, 2, false, true>() : kernel_fn<true, 2, false, false>();
    return stats ? kernel_fn<true, 1, false, true>() : kernel_fn<true, 1, false, false>();
}

// block size and persistent grid for kernel `fn` with `warp_smem` bytes per
// warp after `table_smem` bytes per block (the code table of a mixed launch)
int launch_shape(const void *fn, int table_smem, int warp_smem, int B, int wpb, int *grid_out, int *wpb_out,
                 int *smem_out) {
    int dev = 0, sms = 0, max_smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_status(e);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    while (wpb > 1 && table_smem + wpb * warp_smem > max_smem) wpb >>= 1;
    if (table_smem + wpb * warp_smem > max_smem) return POLAR_ELIMIT;
    const int smem = table_smem + wpb * warp_smem;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_status(e);
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, wpb * 32, smem);
    if (e != cudaSuccess) return cuda_status(e);
    if (per_sm < 1) return POLAR_ELIMIT;
    long long grid = (long long)sms * per_sm;
    const long long want = (long long)(B + wpb - 1) / wpb;
    if (want < grid) grid = want;
    *grid_out = int(grid);
    *wpb_out = wpb;
    *smem_out = smem;
    return 0;
}

cudaError_t launch_fn(const void *fn, int grid, int wpb, int smem, cudaStream_t stream, Args &a) {
    void *args[] = {&a};
    return cudaLaunchKernel(fn, dim3(static_cast<unsigned>(grid)), dim3(static_cast<unsigned>(wpb * 32)), args,
                            size_t(smem), stream);
}

int launch_scs_decode(const polar_plan *p, const DeviceTables *dt, const float *d_llr, int B, int D, int L,
                      uint32_t *d_info, float *d_pm, int8_t *d_status, uint32_t *d_stats, cudaStream_t stream) {
    if (B == 0) return 0;
    Args a{};
    a.code = make_code(p, dt->ops, dt->crc_rows, dt->msg_pos, dt->scales);
    a.D = D;
    a.L = L;
    a.llr = d_llr;
    a.B = B;
    a.info_out = d_info;
    a.pm_out = d_pm;
    a.status_out = d_status;
    a.stats_out = d_stats;
    a.warp_smem = warp_smem_bytes(p->N, p->W, p->nbranch);
    a.llr_vec = ((reinterpret_cast<uintptr_t>(d_llr) & 15u) == 0u) ? 1 : 0;
    a.chunk = 1;
    a.scratch_stride = (long long)(D + 1) * a.code.snap_words;
    int wpb_pref = 4;
    long long deep_fit = 0;
    if (D > POLAR_MAX_D_GPU) {  // the memory stack
        if (p->exact) return POLAR_ELIMIT;
        // one snapshot slot per iteration plus the first complete path; at
        // most 1 + 7 live entries per iteration (a pop, then <= 8 candidates)
        const long long max_iter = (long long)L * (p->nbranch + 9) + 2;
        const long long cap = std::min<long long>(D, 1 + 7 * max_iter);
        a.deep_cap = int(cap);
        a.deep_ent_off = (max_iter + 1) * a.code.snap_words;  // a multiple of 8 words: 16-byte aligned
        a.scratch_stride = a.deep_ent_off + 4 * cap;
        a.deep_best_off = a.warp_smem;
        a.warp_smem = (a.warp_smem + 8 * int((cap + 31) / 32) + 15) & ~15;
        deep_fit = kDeepScratchBytes / (a.scratch_stride * 4);  // warps whose scratch fits the budget
        if (deep_fit < 1) return POLAR_ELIMIT;
        while (wpb_pref > 1 && wpb_pref > deep_fit) wpb_pref >>= 1;
    }

    int grid = 0, wpb = 0, smem = 0;
    const void *fn = uniform_kernel(p, D, d_stats != nullptr);
    int rc = launch_shape(fn, 0, a.warp_smem, B, wpb_pref, &grid, &wpb, &smem);
    if (rc) return rc;
    if (deep_fit > 0 && (long long)grid * wpb > deep_fit) grid = int(deep_fit / wpb);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    const size_t bytes = 64 + size_t(grid) * size_t(wpb) * size_t(a.scratch_stride) * 4;
    void *ws = nullptr;
    keep_pool_memory(dev);
    e = cudaMallocAsync(&ws, bytes, stream);
    if (e != cudaSuccess) return cuda_status(e);
    a.counter = reinterpret_cast<unsigned *>(ws);
    a.scratch = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(ws) + 64);
    e = cudaMemsetAsync(ws, 0, 64, stream);
    if (e == cudaSuccess) {
        e = launch_fn(fn, grid, wpb, smem, stream, a);
    }
    cudaError_t e2 = cudaFreeAsync(ws, stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (e2 != cudaSuccess) return cuda_status(e2);
    return 0;
}

// ---------------------------------------------------------------------------
// Mixed batches: frames of different codes, D and L in one persistent launch
// ---------------------------------------------------------------------------

// device table of the set's codes, made on first use (needs each plan's
// device tables); the caller holds set->mu
static int set_device_codes(const polar_plan_set *set, const Code **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (set->device == dev && set->d_codes) {
        *out = static_cast<const Code *>(set->d_codes);
        return 0;
    }
    if (set->device >= 0) return POLAR_EINVAL;  // a set serves one device
    for (const polar_plan *p : set->plans)
        if (p->exact) return POLAR_EINVAL;  // plan sets decode with min-sum only
    std::vector<Code> codes(set->plans.size());
    for (size_t i = 0; i < set->plans.size(); ++i) {
        const DeviceTables *dt = nullptr;
        int rc = plan_device(set->plans[i], &dt);
        if (rc) return rc;
        codes[i] = make_code(set->plans[i], dt->ops, dt->crc_rows, dt->msg_pos, dt->scales);
    }
    void *d = nullptr;
    e = cudaMalloc(&d, codes.size() * sizeof(Code));
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaMemcpy(d, codes.data(), codes.size() * sizeof(Code), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_status(e);
    }
    set->d_codes = d;
    set->device = dev;
    *out = static_cast<const Code *>(d);
    return 0;
}

void free_set_device(polar_plan_set *set) {
    if (set->d_codes) {
        int cur = -1;
        cudaGetDevice(&cur);
        cudaSetDevice(set->device);
        cudaFree(set->d_codes);
        if (cur >= 0) cudaSetDevice(cur);
    }
    set->d_codes = nullptr;
    set->device = -1;
}

// B claims over d_order (null: frames 0 .. B-1) of a batch of nframes frames
int launch_scs_decode_mixed(const polar_plan_set *set, const int4 *d_frames, const int *d_order, int B, int Dmax,
                            const float *d_llr, const long long *d_llr_off, uint32_t *d_info,
                            const long long *d_info_off, float *d_pm, int8_t *d_status, uint32_t *d_stats,
                            cudaStream_t stream, int wpb_req, int chunk_req, int nframes) {
    if (B == 0) return 0;
    const Code *codes = nullptr;
    int wpb_pref, chunk;
    {
        std::lock_guard<std::mutex> g(set->mu);
        int rc = set_device_codes(set, &codes);
        if (rc) return rc;
        wpb_pref = wpb_req > 0 ? wpb_req : (set->tuned_wpb > 0 ? set->tuned_wpb : 4);
        chunk = chunk_req > 0 ? chunk_req : (set->tuned_chunk > 0 ? set->tuned_chunk : 1);
    }
    Args a{};
    a.codes = codes;
    a.ncodes = int(set->plans.size());
    a.frames = d_frames;
    a.order = d_order;
    a.nframes = nframes;
    a.llr_off = d_llr_off;
    a.info_off = d_info_off;
    a.Dmax = Dmax;
    a.llr = d_llr;
    a.B = B;
    a.info_out = d_info;
    a.pm_out = d_pm;
    a.status_out = d_status;
    a.stats_out = d_stats;
    a.warp_smem = warp_smem_bytes(set->Nmax, set->Wmax, set->nbranch_max);
    a.codes_smem = codes_smem_bytes(a.ncodes);
    a.llr_vec = ((reinterpret_cast<uintptr_t>(d_llr) & 15u) == 0u) ? 1 : 0;
    a.chunk = chunk;
    a.scratch_stride = (long long)(Dmax + 1) * (((set->Wmax + 4) + 7) & ~7);

    int grid = 0, wpb = 0, smem = 0;
    const int nb_units = (B + chunk - 1) / chunk;
    const void *fn = mixed_kernel(Dmax, d_stats != nullptr);
    int rc = launch_shape(fn, a.codes_smem, a.warp_smem, nb_units, wpb_pref, &grid, &wpb, &smem);
    if (rc) return rc;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    const size_t bytes = 64 + size_t(grid) * size_t(wpb) * size_t(a.scratch_stride) * 4;
    void *ws = nullptr;
    keep_pool_memory(dev);
    e = cudaMallocAsync(&ws, bytes, stream);
    if (e != cudaSuccess) return cuda_status(e);
    a.counter = reinterpret_cast<unsigned *>(ws);
    a.scratch = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(ws) + 64);
    e = cudaMemsetAsync(ws, 0, 64, stream);
    if (e == cudaSuccess) {
        e = launch_fn(fn, grid, wpb, smem, stream, a);
    }
    cudaError_t e2 = cudaFreeAsync(ws, stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (e2 != cudaSuccess) return cuda_status(e2);
    return 0;
}

// ---------------------------------------------------------------------------
// Served requests: the persistent kernel of the continuous-batching engine
// ---------------------------------------------------------------------------
int serve_codes(const polar_plan_set *set, const void **out) {
    std::lock_guard<std::mutex> g(set->mu);
    const Code *c = nullptr;
    int rc = set_device_codes(set, &c);
    *out = c;
    return rc;
}

int launch_scs_serve(const polar_plan_set *set, const void *codes_v, const int4 *d_frames, int B, int Dmax,
                     const float *d_arena, const long long *d_llr_off, uint32_t *d_info, const long long *d_info_off,
                     float *d_pm, int8_t *d_status, const unsigned long long *d_head, const int *h_abort,
                     unsigned char *h_done, unsigned long long *d_t_done, unsigned long long *d_t_start, int *d_error,
                     unsigned long long wait_ns, unsigned *d_counter, uint32_t *d_scratch, size_t scratch_bytes,
                     int wpb_pref, cudaStream_t stream) {
    const Code *codes = static_cast<const Code *>(codes_v);
    Args a{};
    a.codes = codes;
    a.ncodes = int(set->plans.size());
    a.frames = d_frames;
    a.llr_off = d_llr_off;
    a.info_off = d_info_off;
    a.Dmax = Dmax;
    a.llr = d_arena;
    a.B = B;
    a.info_out = d_info;
    a.pm_out = d_pm;
    a.status_out = d_status;
    a.warp_smem = warp_smem_bytes(set->Nmax, set->Wmax, set->nbranch_max);
    a.codes_smem = codes_smem_bytes(a.ncodes);
    a.llr_vec = 1;  // requests are decoded from 16-byte aligned staging copies
    a.chunk = 1;
    a.serve_stage_off = (long long)(Dmax + 1) * (((set->Wmax + 4) + 7) & ~7);
    a.scratch_stride = a.serve_stage_off + ((set->Nmax + 3) & ~3);
    a.head = d_head;
    a.abort_flag = h_abort;
    a.done_flag = h_done;
    a.t_done = d_t_done;
    a.t_start = d_t_start;
    a.error_flag = d_error;
    a.wait_ns = wait_ns;
    a.counter = d_counter;
    a.scratch = d_scratch;
    int dev = 0, sms = 0, max_smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int wpb = wpb_pref > 0 ? wpb_pref : 4;
    while (wpb > 1 && a.codes_smem + wpb * a.warp_smem > max_smem) wpb >>= 1;
    if (a.codes_smem + wpb * a.warp_smem > max_smem) return POLAR_ELIMIT;
    const int smem = a.codes_smem + wpb * a.warp_smem;
    const void *kern = Dmax <= 32 ? reinterpret_cast<const void *>(scs_serve_kernel<1>)
                                  : reinterpret_cast<const void *>(scs_serve_kernel<2>);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_status(e);
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, wpb * 32, smem);
    if (e != cudaSuccess) return cuda_status(e);
    if (per_sm < 1) return POLAR_ELIMIT;
    long long grid = (long long)sms * per_sm;
    const size_t per_block = size_t(wpb) * size_t(a.scratch_stride) * 4;
    if (size_t(grid) * per_block > scratch_bytes) grid = (long long)(scratch_bytes / per_block);
    if (grid < 1) return POLAR_ENOMEM;
    if (Dmax <= 32) scs_serve_kernel<1><<<unsigned(grid), unsigned(wpb * 32), size_t(smem), stream>>>(a);
    else scs_serve_kernel<2><<<unsigned(grid), unsigned(wpb * 32), size_t(smem), stream>>>(a);
    e = cudaGetLastError();
    return e == cudaSuccess ? 0 : cuda_status(e);
}

size_t serve_scratch_bytes(const polar_plan_set *set, int Dmax) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t stride = (size_t(Dmax + 1) * size_t(((set->Wmax + 4) + 7) & ~7) + size_t((set->Nmax + 3) & ~3)) * 4;
    return size_t(sms > 0 ? sms : 1) * 8 * 4 * stride;  // at most 8 blocks of 4 warps per SM
}

int read_device_ns(unsigned long long *d_out, cudaStream_t s) {
    read_global_ns<<<1, 1, 0, s>>>(d_out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 0 : cuda_status(e);
}

// ---------------------------------------------------------------------------
// Decoding without any allocation by the library.
//
// Some callers cannot allocate device memory when they decode: code that runs
// under a fixed memory budget reserved at start-up, real-time loops where
// cudaMalloc/cudaMallocAsync may block or fail, or processes whose device
// memory is owned by another allocator.  For them scs_decode_batch_noalloc
// keeps the decoder's scratch (the per-warp beta snapshots and the frame
// counter) and its copy of the plan's tables in two fixed file-scope device
// arrays below.  Every GPU that loads the library holds these arrays (16 MiB
// + 1 MiB) until the process exits.
//
// The host needs their device addresses: in host code the names are host-side
// stand-ins, so they are fetched once per device with cudaGetSymbolAddress,
// with that device current, on the first call made on that device.  The
// table area remembers which plan (serial number and version) it holds, so a
// call with the same plan issues no copy at all.
// ---------------------------------------------------------------------------
constexpr size_t kStaticScratchBytes = size_t(16) << 20;
constexpr size_t kStaticTableBytes = size_t(1) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];
static __device__ __align__(256) unsigned char g_static_tables[kStaticTableBytes];

namespace {

struct StaticAreas {
    bool ready = false;
    void *scratch = nullptr;
    void *tables = nullptr;
    uint64_t serial = 0, version = 0;  // plan whose tables the area holds (0: none)
};
std::mutex g_static_mu;
StaticAreas g_static_areas[64];

int static_areas(int dev, StaticAreas *out) {
    if (dev < 0 || dev >= 64) return POLAR_EINVAL;
    std::lock_guard<std::mutex> g(g_static_mu);
    StaticAreas &s = g_static_areas[dev];
    if (!s.ready) {
        void *scr = nullptr, *tab = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&scr, g_static_scratch);
        if (e != cudaSuccess) return cuda_status(e);
        e = cudaGetSymbolAddress(&tab, g_static_tables);
        if (e != cudaSuccess) return cuda_status(e);
        s.scratch = scr;
        s.tables = tab;
        s.ready = true;
    }
    *out = s;
    return 0;
}

// record which plan's tables the device's table area holds (serial 0: none)
void static_tables_hold(int dev, uint64_t serial, uint64_t version) {
    std::lock_guard<std::mutex> g(g_static_mu);
    g_static_areas[dev].serial = serial;
    g_static_areas[dev].version = version;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

int launch_scs_decode_noalloc(const polar_plan *p, const float *d_llr, int B, int D, int L, uint32_t *d_info,
                              float *d_pm, int8_t *d_status, uint32_t *d_stats, cudaStream_t stream) {
    if (B == 0) return 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    StaticAreas areas;
    int rc = static_areas(dev, &areas);
    if (rc) return rc;
    // the plan's tables and sizes are read under its lock (polar_plan_set_scales
    // may replace the scales on another thread)
    std::lock_guard<std::mutex> plan_lock(p->mu);

    // layout of the plan's tables in the static table area
    const size_t ops_bytes = p->dev_ops.size() * sizeof(KOp);
    const size_t rows_off = align_up(ops_bytes, 256);
    const size_t rows_bytes = p->crc_rows.size() * sizeof(uint32_t);
    const size_t pos_off = align_up(rows_off + rows_bytes, 256);
    const size_t pos_bytes = p->msg_pos.size() * sizeof(uint16_t);
    const size_t sc_off = align_up(pos_off + pos_bytes, 256);
    const size_t sc_bytes = p->scales.size() * sizeof(float);
    if (sc_off + sc_bytes > kStaticTableBytes) return POLAR_ESCRATCH;
    unsigned char *tab = static_cast<unsigned char *>(areas.tables);

    Args a{};
    a.code = make_code(p, reinterpret_cast<const KOp *>(tab), reinterpret_cast<const uint32_t *>(tab + rows_off),
                       reinterpret_cast<const uint16_t *>(tab + pos_off), reinterpret_cast<const float *>(tab + sc_off));
    a.D = D;
    a.L = L;
    a.llr = d_llr;
    a.B = B;
    a.info_out = d_info;
    a.pm_out = d_pm;
    a.status_out = d_status;
    a.stats_out = d_stats;
    a.warp_smem = warp_smem_bytes(p->N, p->W, p->nbranch);
    a.llr_vec = ((reinterpret_cast<uintptr_t>(d_llr) & 15u) == 0u) ? 1 : 0;
    a.chunk = 1;
    a.scratch_stride = (long long)(D + 1) * a.code.snap_words;

    // as many resident warps as the static scratch holds (the kernel is
    // persistent and claims frames dynamically, so fewer warps only cost speed)
    const size_t per_warp = size_t(a.scratch_stride) * 4;
    const size_t warps_fit = (kStaticScratchBytes - 64) / per_warp;
    if (warps_fit < 1) return POLAR_ESCRATCH;
    int wpb = 4;
    while (wpb > 1 && size_t(wpb) > warps_fit) wpb >>= 1;
    int grid = 0, smem = 0;
    const void *fn = uniform_kernel(p, D, d_stats != nullptr);
    rc = launch_shape(fn, 0, a.warp_smem, B, wpb, &grid, &wpb, &smem);
    if (rc) return rc;
    const long long fit = (long long)(warps_fit / size_t(wpb));
    if (fit < grid) grid = int(fit);

    a.counter = static_cast<unsigned *>(areas.scratch);
    a.scratch = reinterpret_cast<uint32_t *>(static_cast<unsigned char *>(areas.scratch) + 64);
    // the tables, unless this plan's current version is already in the area;
    // they come from the plan's pageable host vectors, a copy for which CUDA
    // may first wait on the host for earlier work on the stream
    if (areas.serial != p->serial || areas.version != p->version) {
        static_tables_hold(dev, 0, 0);  // in flux until every copy is issued
        e = cudaMemcpyAsync(tab, p->dev_ops.data(), ops_bytes, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess && rows_bytes)
            e = cudaMemcpyAsync(tab + rows_off, p->crc_rows.data(), rows_bytes, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess && pos_bytes)
            e = cudaMemcpyAsync(tab + pos_off, p->msg_pos.data(), pos_bytes, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess && sc_bytes)
            e = cudaMemcpyAsync(tab + sc_off, p->scales.data(), sc_bytes, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return cuda_status(e);
        static_tables_hold(dev, p->serial, p->version);
    }
    // the frame counter back to zero (the array keeps whatever the previous
    // call left in it)
    e = cudaMemsetAsync(areas.scratch, 0, 64, stream);
    if (e != cudaSuccess) return cuda_status(e);
    e = launch_fn(fn, grid, wpb, smem, stream, a);
    return e == cudaSuccess ? 0 : cuda_status(e);
}

}  // namespace polarscs

#ifdef POLAR_PHASE_TIMERS
// debug builds only: read (and optionally clear) the per-phase cycle sums
extern "C" int polar_phase_cycles(unsigned long long *out, int reset) {
    cudaError_t e = cudaMemcpyFromSymbol(out, polarscs::g_phase_cycles, sizeof(unsigned long long) * polarscs::PH_N);
    if (e == cudaSuccess && reset) {
        static const unsigned long long zeros[polarscs::PH_N] = {};
        e = cudaMemcpyToSymbol(polarscs::g_phase_cycles, zeros, sizeof(zeros));
    }
    return e == cudaSuccess ? polarscs::PH_N : -3;
}
#endif
