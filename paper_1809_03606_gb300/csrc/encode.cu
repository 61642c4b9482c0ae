// encode.cu - batched polar encoding c = u F^{(x)n} (Sec. 2.1, Fig. encoder)
// with the CRC of the plan appended to the message; systematic codes
// (Sec. 2.2.2) take a second pass of the XOR tree after the frozen
// positions of the first pass's output are cleared.
//
// One warp per frame: the message bits are scattered onto the information
// set in a packed shared-memory row, the CRC register is the XOR of the
// registers of the set message bits (the long division is linear), and the
// n stages of the XOR tree run as shift/mask steps inside 32-bit words and
// as word XORs across words.
#include <cuda_runtime.h>

#include <cstdint>

#include "plan.h"

namespace polarscs {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;

struct EncArgs {
    const uint32_t *msg;
    uint32_t *cw;
    int B, N, W, Kmsg, crc, msg_words;
    const uint16_t *info_pos;
    const uint32_t *crc_contrib;
    const uint32_t *info_bits;  // W words, information positions (systematic pass)
    int systematic;
};

// u <- u F^{(x)n} on the warp's packed row: shift/mask stages inside words,
// word XORs across words
__device__ void xor_tree(uint32_t *u, int N, int W, int lane) {
    for (int k = lane; k < W; k += 32) {
        uint32_t x = u[k];
        if (N > 1) x ^= (x >> 1) & 0x55555555u;
        if (N > 2) x ^= (x >> 2) & 0x33333333u;
        if (N > 4) x ^= (x >> 4) & 0x0F0F0F0Fu;
        if (N > 8) x ^= (x >> 8) & 0x00FF00FFu;
        if (N > 16) x ^= (x >> 16) & 0x0000FFFFu;
        if (N < 32) x &= (1u << N) - 1u;
        u[k] = x;
    }
    __syncwarp();
    for (int hw = 1; hw < W; hw <<= 1) {
        for (int k = lane; k < W; k += 32)
            if (!(k & hw)) u[k] ^= u[k + hw];
        __syncwarp();
    }
}

__global__ void __launch_bounds__(128) polar_encode_kernel(EncArgs a) {
    extern __shared__ uint32_t esm[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint32_t *u = esm + size_t(wib) * a.W;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int b = blockIdx.x * (blockDim.x >> 5) + wib; b < a.B; b += warps) {
        const uint32_t *m = a.msg + size_t(b) * a.msg_words;
        for (int k = lane; k < a.W; k += 32) u[k] = 0u;
        __syncwarp();
        uint32_t reg = 0u;
        for (int j = lane; j < a.Kmsg; j += 32) {
            if ((m[j >> 5] >> (j & 31)) & 1u) {
                const int p = a.info_pos[j];
                atomicOr(&u[p >> 5], 1u << (p & 31));
                if (a.crc) reg ^= __ldg(a.crc_contrib + j);
            }
        }
        if (a.crc) {
            reg = __reduce_xor_sync(FULL, reg);
            for (int r = lane; r < a.crc; r += 32) {
                if ((reg >> (a.crc - 1 - r)) & 1u) {
                    const int p = a.info_pos[a.Kmsg + r];
                    atomicOr(&u[p >> 5], 1u << (p & 31));
                }
            }
        }
        __syncwarp();
        xor_tree(u, a.N, a.W, lane);
        if (a.systematic) {
            for (int k = lane; k < a.W; k += 32) u[k] &= __ldg(a.info_bits + k);
            __syncwarp();
            xor_tree(u, a.N, a.W, lane);
        }
        uint32_t *c = a.cw + size_t(b) * a.W;
        for (int k = lane; k < a.W; k += 32) c[k] = u[k];
        __syncwarp();
    }
}

}  // namespace

int launch_polar_encode(const polar_plan *p, const DeviceTables *dt, const uint32_t *d_msg, int B, uint32_t *d_cw,
                        cudaStream_t stream) {
    if (B == 0) return 0;
    EncArgs a{d_msg, d_cw, B, p->N, p->W, p->Kmsg, p->crc, (p->Kmsg + 31) / 32, dt->info_pos, dt->crc_contrib,
              dt->info_bits, p->systematic};
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int wpb = 4;
    long long grid = (long long)(B + wpb - 1) / wpb;
    const long long cap = (long long)(sms > 0 ? sms : 1) * 16;
    if (grid > cap) grid = cap;
    const size_t smem = size_t(wpb) * size_t(p->W) * 4;
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(polar_encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return cuda_status(e);
    }
    polar_encode_kernel<<<unsigned(grid), unsigned(wpb * 32), smem, stream>>>(a);
    e = cudaGetLastError();
    return e == cudaSuccess ? 0 : cuda_status(e);
}

}  // namespace polarscs
