// plan.cpp - host-side code construction and decoding-plan builder.
//
// The schedule follows Sec. 3.1 (Fig. fsscsch): the decoding tree of Fig.
// scdectree is walked once per code; a node that the fast simplified scheme
// of Sec. 2.2.2 recognises is decoded by one node operation, any other node
// is split into alpha(left child), <left>, alpha(right child), <right>,
// beta(right child).  Each entry also records where a path that resumes at
// it must have valid alpha (the spine recomputed after a path switch, Sec.
// 3.3 Alg. calp), and the visit-counter index of each branching node (Sec.
// 2.2.5).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>

#include "plan.h"

namespace polarscs {

uint32_t crc_polynomial(int crc) {
    switch (crc) {
    case 8: return 0x07u;
    case 16: return 0x1021u;
    case 24: return 0xB2B117u;
    default: return 0u;
    }
}

static bool pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

int validate_code(int N, int K, const uint8_t *frozen, int crc) {
    if (!pow2(N) || N < 2 || N > (1 << 15)) return POLAR_EINVAL;
    if (K < 1 || K > N) return POLAR_EINVAL;
    if (crc != 0 && crc_polynomial(crc) == 0u) return POLAR_EINVAL;
    if (crc < 0 || crc >= K) return POLAR_EINVAL;
    if (frozen) {
        int nf = 0;
        for (int i = 0; i < N; ++i) nf += frozen[i] ? 1 : 0;
        if (nf != N - K) return POLAR_EINVAL;
    }
    return 0;
}

namespace {

struct Builder {
    const uint8_t *fr;
    int fast;
    std::vector<KOp> ops;
    int nbranch = 0;

    // number of frozen leaves in [s, s + len)
    int frozen_count(int s, int len) const {
        int c = 0;
        for (int i = 0; i < len; ++i) c += fr[s + i] ? 1 : 0;
        return c;
    }

    uint32_t node_kind(int lam, int s) const {
        const int len = 1 << lam;
        if (lam == 0) return fr[s] ? OP_LEAF0 : OP_LEAF1;
        if (!fast) return 0xFFu;
        const int nf = frozen_count(s, len);
        if (nf == len) return OP_R0;
        if (nf == 0) return OP_R1;
        if (nf == len - 1 && !fr[s + len - 1]) return OP_REP;
        if (lam >= 2 && nf == 1 && fr[s]) return OP_SPC;
        return 0xFFu;  // split
    }

    void emit(uint32_t code, int lam, int s) {
        KOp op{code | (uint32_t(lam) << 8), uint32_t(s), NO_TARGET, 0u};
        if (code >= OP_BRANCH) op.w = uint32_t(nbranch++);
        ops.push_back(op);
    }

    void walk(int lam, int s) {
        const uint32_t kind = node_kind(lam, s);
        if (kind != 0xFFu) {
            emit(kind, lam, s);
            return;
        }
        const int half = 1 << (lam - 1);
        emit(OP_F, lam - 1, s);
        walk(lam - 1, s);
        emit(OP_G, lam - 1, s + half);
        walk(lam - 1, s + half);
        emit(OP_COMB, lam - 1, s + half);
    }
};

}  // namespace

}  // namespace polarscs

using namespace polarscs;

extern "C" int polar_construct(int N, int K, float design_snr_db, uint8_t *frozen) {
    if (!frozen || !pow2(N) || N < 2 || N > (1 << 15) || K < 1 || K > N) return POLAR_EINVAL;
    // ln z of every leaf, root first, split top-down in natural leaf order
    std::vector<double> lz(size_t(N), 0.0);
    lz[0] = -(double(K) / double(N)) * std::pow(10.0, double(design_snr_db) / 10.0);
    for (int len = N; len >= 2; len >>= 1) {
        const int half = len >> 1;
        for (int s = 0; s < N; s += len) {
            const double v = lz[size_t(s)];
            const double z = std::exp(v);
            lz[size_t(s)] = v + std::log(2.0) + std::log1p(-0.5 * z);  // ln(2z - z^2)
            lz[size_t(s + half)] = v + v;                               // ln(z^2)
        }
    }
    std::vector<int> idx(static_cast<size_t>(N));
    for (int i = 0; i < N; ++i) idx[size_t(i)] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) {
        if (lz[size_t(a)] != lz[size_t(b)]) return lz[size_t(a)] < lz[size_t(b)];
        return a > b;  // equal parameter: higher index is information
    });
    std::memset(frozen, 1, size_t(N));
    for (int k = 0; k < K; ++k) frozen[idx[size_t(k)]] = 0;
    return 0;
}

extern "C" int polar_plan_create(int N, int K, const uint8_t *frozen, int fast_nodes, int crc, polar_plan **out) {
    if (!out || !frozen) return POLAR_EINVAL;
    *out = nullptr;
    int rc = validate_code(N, K, frozen, crc);
    if (rc) return rc;
    polar_plan *p = new (std::nothrow) polar_plan();
    if (!p) return POLAR_ENOMEM;
    static std::atomic<uint64_t> next_serial{1};
    p->serial = next_serial.fetch_add(1);
    try {
        p->N = N;
        p->n = 0;
        while ((1 << p->n) < N) ++p->n;
        p->K = K;
        p->crc = crc;
        p->Kmsg = K - crc;
        p->fast = fast_nodes ? 1 : 0;
        p->W = N < 32 ? 1 : N / 32;
        p->frozen.assign(frozen, frozen + N);
        for (auto &b : p->frozen) b = b ? 1 : 0;

        Builder bld{p->frozen.data(), p->fast, {}, 0};
        bld.walk(p->n, 0);
        p->ops = std::move(bld.ops);
        p->nbranch = bld.nbranch;

        // alpha restore target of every resume point t: the node whose alpha
        // the first alpha-reading op at or after t reads (the parent of an F/G
        // child, or the node of a node op); the root's alpha is the channel.
        const int nops = int(p->ops.size());
        uint32_t next = NO_TARGET;
        for (int t = nops - 1; t >= 0; --t) {
            const uint32_t code = p->ops[size_t(t)].x & 0xFFu;
            const uint32_t lam = (p->ops[size_t(t)].x >> 8) & 0xFFu;
            const uint32_t s = p->ops[size_t(t)].y;
            if (code == OP_F || code == OP_G) {
                const uint32_t plam = lam + 1;
                const uint32_t ps = s & ~((1u << plam) - 1u);
                next = (int(plam) >= p->n) ? NO_TARGET : (plam | (ps << 8));
            } else if (code != OP_COMB) {  // a node op reads its own alpha
                next = (int(lam) >= p->n) ? NO_TARGET : (lam | (s << 8));
            }
            p->ops[size_t(t)].z = next;
        }

        // the kernels' schedule: COMB runs and alpha descents merged into one
        // entry (a path resumes only right after a branching operation, i.e.
        // at the start of a run, so every resume point survives the merge)
        for (int t = 0; t < nops;) {
            KOp o = p->ops[size_t(t)];
            const uint32_t code = o.x & 0xFFu;
            const int lam = int((o.x >> 8) & 0xFFu);
            const uint32_t s = o.y;
            int k = 1;
            auto at = [&](int q, uint32_t c, int l, uint32_t st) {
                const KOp &n = p->ops[size_t(q)];
                return (n.x & 0xFFFFu) == (c | uint32_t(l) << 8) && n.y == st;
            };
            if (code == OP_COMB) {
                uint32_t st = s;
                while (t + k < nops && k < 256 && lam + k < 32 && (st >= (1u << (lam + k - 1))) &&
                       at(t + k, OP_COMB, lam + k, st - (1u << (lam + k - 1)))) {
                    st -= 1u << (lam + k - 1);
                    ++k;
                }
            } else if (code == OP_F || code == OP_G) {
                while (t + k < nops && k < 256 && lam - k >= 0 && at(t + k, OP_F, lam - k, s)) ++k;
            }
            o.x |= uint32_t(k - 1) << 16;
            p->dev_ops.push_back(o);
            t += k;
        }

        // information and message positions
        for (int i = 0; i < N; ++i)
            if (!p->frozen[size_t(i)]) p->info_pos.push_back(uint16_t(i));
        p->msg_pos.assign(p->info_pos.begin(), p->info_pos.begin() + p->Kmsg);
        p->info_mask.assign(size_t(N), 0u);
        p->info_bits.assign(size_t(p->W), 0u);
        for (int i = 0; i < N; ++i) {
            p->info_mask[size_t(i)] = p->frozen[size_t(i)] ? 0u : 1u;
            if (!p->frozen[size_t(i)]) p->info_bits[size_t(i >> 5)] |= 1u << (i & 31);
        }

        // CRC register of each unit message (linearity of the long division)
        if (crc) {
            const uint32_t poly = crc_polynomial(crc);
            const uint32_t mask = (crc == 32) ? 0xFFFFFFFFu : ((1u << crc) - 1u);
            const uint32_t top = 1u << (crc - 1);
            p->crc_contrib.assign(size_t(p->Kmsg), 0u);
            uint32_t reg = poly & mask;  // a single 1 as the last message bit
            for (int m = p->Kmsg - 1; m >= 0; --m) {
                p->crc_contrib[size_t(m)] = reg;
                const bool fb = (reg & top) != 0;
                reg = (reg << 1) & mask;
                if (fb) reg ^= poly;
            }
            build_crc_rows(p);
        }
    } catch (...) {
        delete p;
        return POLAR_ENOMEM;
    }
    *out = p;
    return 0;
}

namespace polarscs {

// Syndrome rows over codeword bits.  Non-systematic: codeword bit q reaches
// u_j for every j whose bits are a subset of q's (u = x F^{(x)n}, an
// involution), and u_j on the information set is message bit rank(j).
// Systematic: information bit k is codeword bit info_pos[k] itself.
void build_crc_rows(polar_plan *p) {
    const int N = p->N, K = p->K, crc = p->crc;
    p->crc_rows.assign(size_t(crc) * size_t(p->W), 0u);
    if (!crc) return;
    std::vector<int> info_rank(size_t(N), -1);
    for (int k = 0; k < K; ++k) info_rank[p->info_pos[size_t(k)]] = k;
    auto unit = [&](int k) -> uint32_t {  // syndrome of information bit k alone
        return k < p->Kmsg ? p->crc_contrib[size_t(k)] : (1u << (crc - 1 - (k - p->Kmsg)));
    };
    for (int q = 0; q < N; ++q) {
        uint32_t syn = 0;
        if (p->systematic) {
            if (info_rank[size_t(q)] >= 0) syn = unit(info_rank[size_t(q)]);
        } else {
            for (int j = q;; j = (j - 1) & q) {  // all submasks of q
                const int k = info_rank[size_t(j)];
                if (k >= 0) syn ^= unit(k);
                if (j == 0) break;
            }
        }
        for (int r = 0; r < crc; ++r)
            if ((syn >> r) & 1u) p->crc_rows[size_t(r) * size_t(p->W) + size_t(q >> 5)] |= 1u << (q & 31);
    }
}

namespace {

// x <- x F^{(x)n} on a packed N-bit row (the XOR tree of Sec. 2.1)
void xor_tree(std::vector<uint64_t> &w, int N) {
    static const uint64_t lo[6] = {0x5555555555555555ull, 0x3333333333333333ull, 0x0F0F0F0F0F0F0F0Full,
                                   0x00FF00FF00FF00FFull, 0x0000FFFF0000FFFFull, 0x00000000FFFFFFFFull};
    for (int st = 0; (1 << st) < N && st < 6; ++st)
        for (auto &x : w) x ^= (x >> (1 << st)) & lo[st];
    const int nw = int(w.size());
    for (int h = 1; h < nw; h <<= 1)
        for (int k = 0; k < nw; ++k)
            if (!(k & h)) w[size_t(k)] ^= w[size_t(k + h)];
}

// the two-pass encoder (x = F(clear_frozen(F(v))), v the information bits
// placed on A) is systematic iff it maps every unit information vector to
// itself on A; both passes are linear, so unit vectors suffice
bool two_pass_is_systematic(const polar_plan *p) {
    const int N = p->N, nw = (N + 63) / 64;
    std::vector<uint64_t> mask(static_cast<size_t>(nw), 0ull), w(static_cast<size_t>(nw), 0ull);
    for (int i = 0; i < N; ++i)
        if (!p->frozen[size_t(i)]) mask[size_t(i >> 6)] |= 1ull << (i & 63);
    for (int k = 0; k < p->K; ++k) {
        const int a = p->info_pos[size_t(k)];
        std::fill(w.begin(), w.end(), 0ull);
        w[size_t(a >> 6)] = 1ull << (a & 63);
        xor_tree(w, N);
        for (int q = 0; q < nw; ++q) w[size_t(q)] &= mask[size_t(q)];
        xor_tree(w, N);
        for (int q = 0; q < nw; ++q) {
            const uint64_t want = (q == (a >> 6)) ? (1ull << (a & 63)) : 0ull;
            if ((w[size_t(q)] & mask[size_t(q)]) != want) return false;
        }
    }
    return true;
}

}  // namespace
}  // namespace polarscs

extern "C" int polar_plan_set_exact(polar_plan *p, int on) {
    if (!p) return POLAR_EINVAL;
    std::lock_guard<std::mutex> g(p->mu);
    if (p->dev.device >= 0) return POLAR_EINVAL;  // tables already on a device
    if (on && (p->fast || !p->scales.empty())) return POLAR_EINVAL;
    p->exact = on ? 1 : 0;
    ++p->version;
    return 0;
}

extern "C" int polar_plan_set_systematic(polar_plan *p, int on) {
    if (!p) return POLAR_EINVAL;
    std::lock_guard<std::mutex> g(p->mu);
    if (p->dev.device >= 0) return POLAR_EINVAL;  // tables already on a device
    try {
        if (on && !polarscs::two_pass_is_systematic(p)) return POLAR_EINVAL;
        p->systematic = on ? 1 : 0;
        ++p->version;
        polarscs::build_crc_rows(p);
    } catch (...) {
        return POLAR_ENOMEM;
    }
    return 0;
}

extern "C" int polar_plan_schedule(const polar_plan *p, int32_t *ops_out, int max_ops) {
    if (!p || (max_ops > 0 && !ops_out)) return POLAR_EINVAL;
    const int nops = int(p->ops.size());
    for (int t = 0; t < nops && t < max_ops; ++t) {
        const uint32_t code = p->ops[size_t(t)].x & 0xFFu;
        const int lam = int((p->ops[size_t(t)].x >> 8) & 0xFFu);
        const int phi = int(p->ops[size_t(t)].y >> lam);
        int32_t o;
        switch (code) {
        case OP_F:
        case OP_G: o = 0; break;
        case OP_COMB: o = 1; break;
        case OP_R0: o = 2; break;
        case OP_R1: o = 3; break;
        case OP_REP: o = 4; break;
        case OP_SPC: o = 5; break;
        case OP_LEAF0: o = 6; break;
        default: o = 7; break;
        }
        ops_out[3 * t] = o;
        ops_out[3 * t + 1] = lam;
        ops_out[3 * t + 2] = phi;
    }
    return nops;
}
