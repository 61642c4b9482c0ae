// plan.h - internal plan representation shared by the library's translation
// units (host builder, kernels, C ABI).  Not part of the public interface.
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <vector>

#include "polarscs.h"

namespace polarscs {

// Kernel operation codes.  alpha ops of Eq. llrcalc are split into F (even
// child, min-sum f) and G (odd child, g); COMB is the in-place beta operation
// of Sec. 4.  Codes >= OP_BRANCH create several candidate paths.
enum OpCode : uint32_t {
    OP_F = 0,
    OP_G = 1,
    OP_COMB = 2,
    OP_R0 = 3,
    OP_LEAF0 = 4,
    OP_LEAF1 = 5,  // first branching code
    OP_REP = 6,
    OP_R1 = 7,
    OP_SPC = 8,
};
constexpr uint32_t OP_BRANCH = OP_LEAF1;
constexpr uint32_t NO_TARGET = 0xFFFFFFFFu;

// One schedule entry, 16 bytes, read by every lane of a warp (broadcast).
//  x: code | lambda << 8      (lambda of the node the op writes / decodes)
//  y: first leaf s of that node
//  z: alpha restore target for a path resuming at this op: the node whose
//     alpha the next alpha-reading op needs, as lambda | s << 8, or NO_TARGET
//  w: branching ordinal (index of the visit counter) for codes >= OP_BRANCH
// The kernels read the schedule with runs merged (polar_plan::dev_ops): bits
// 16..23 of x hold run - 1, where a COMB run climbs one stage per step (the
// next odd child starts 2^lambda leaves earlier) and an alpha run is an F or
// G followed by F ops one stage lower each (same first leaf).
struct alignas(16) KOp {
    uint32_t x, y, z, w;
};

struct DeviceTables {
    int device = -1;
    KOp *ops = nullptr;
    uint32_t *crc_rows = nullptr;    // crc x W words: syndrome bit r over codeword bits
    uint16_t *msg_pos = nullptr;     // Kmsg information indices of the message bits
    uint16_t *info_pos = nullptr;    // K information indices
    uint32_t *crc_contrib = nullptr; // Kmsg CRC registers of unit messages
    uint8_t *info_mask = nullptr;    // N bytes: 1 = information leaf
    uint32_t *info_bits = nullptr;   // W words: information positions, packed
    float *scales = nullptr;         // n per-stage f scales, or null (unscaled)
};

}  // namespace polarscs

struct polar_plan {
    int N = 0, n = 0, K = 0, Kmsg = 0, crc = 0, fast = 0;
    int W = 0;        // 32-bit words of a packed N-bit array (at least 1)
    int nbranch = 0;  // branching operations (visit counters)
    std::vector<uint8_t> frozen;
    std::vector<polarscs::KOp> ops;      // the schedule, one entry per operation
    std::vector<polarscs::KOp> dev_ops;  // the kernels' schedule: runs merged
    std::vector<uint32_t> crc_rows;
    std::vector<uint16_t> msg_pos, info_pos;
    std::vector<uint32_t> crc_contrib;
    std::vector<uint8_t> info_mask;
    std::vector<float> scales;  // empty: unscaled min-sum
    std::vector<uint32_t> info_bits;  // W words: 1 = information position
    int systematic = 0;               // codeword carries the information bits
    int exact = 0;                    // exact-f decoding (box-plus f, exact leaf metric)
    // identity of the plan's tables: a process-wide serial number given at
    // creation and a version bumped (under mu) by every call that changes
    // them; lets a copy of the tables on a device be recognised as current
    uint64_t serial = 0, version = 0;
    mutable std::mutex mu;
    mutable polarscs::DeviceTables dev;
};

// A set of plans decoded together by scs_decode_mixed (frames name their
// plan by index).  Device state is made on first use and serves one device.
struct polar_plan_set {
    std::vector<const polar_plan *> plans;
    int Nmax = 0, Wmax = 0, nbranch_max = 0;
    mutable std::mutex mu;
    mutable int device = -1;
    mutable void *d_codes = nullptr;  // device array of the kernels' code records
    mutable int tuned_wpb = 0, tuned_chunk = 0;  // 0: not tuned yet
};

namespace polarscs {

// An NVTX range over the lifetime of the object (host side): every C ABI
// entry point that launches work names itself, so a trace (nsys, ncu --nvtx)
// shows which call issued which kernels.  Without an attached tool the calls
// return at once.
struct TraceRange {
    explicit TraceRange(const char *name);
    ~TraceRange();
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

int validate_code(int N, int K, const uint8_t *frozen, int crc);
// CRC syndrome rows over codeword bits for the plan's encoding (needs
// info_pos, crc_contrib).
void build_crc_rows(polar_plan *p);
uint32_t crc_polynomial(int crc);
// Upload the plan's tables to the current device (once).  Returns 0 or an error.
int plan_device(const polar_plan *plan, const DeviceTables **out);
int cuda_status(int err);  // map a cudaError_t to POLAR_ECUDA / POLAR_ENOMEM
void keep_pool_memory(int dev);

}  // namespace polarscs
