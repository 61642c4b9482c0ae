/*
 * polar_oracle.c - plain, slow, scalar CPU oracle for successive-cancellation
 * stack (SCS) decoding of polar codes, written from Aurora & Gross, "Towards
 * Practical Software Stack Decoding of Polar Codes" (arXiv 1809.03606).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the bench's CPU
 * baseline may load this file; the GPU library never calls it and shares no
 * code, table or header with it.
 *
 * Build flags: -O2 -fno-fast-math -ffp-contract=off.  All single-precision
 * arithmetic happens in the order written here (no FMA contraction), so the
 * results are reproducible bit for bit.
 *
 * Paper notation: a node of the decoding tree is (lambda, phi) with
 * Lambda = 2^lambda leaves starting at leaf s = phi * Lambda (Sec. 2.1,
 * Sec. 2.2.1).  Stage n is the root, whose LLRs are the channel LLRs (Eq.
 * llrcalc).  Where the paper is silent or garbled this file follows these
 * readings (each one is listed with its justification in the design notes):
 *   R1  g(a, b, beta) = b + (1 - 2 beta) a, with a = alpha_p[i],
 *       b = alpha_p[i + Lambda]  (Fig. minsum; the printed Eq. minsum swaps
 *       the operands).
 *   R2  HD(x) = (x < 0), so HD(-0) = 0; the sign of f is the XOR of the sign
 *       bits of its operands.
 *   R3  Alg. calp: psi = floor(phi / 2), loop index i = 0 .. Lambda-1.
 *   R6  Fast-node precedence R-0 > R-1 > REP > SPC; REP needs Lambda >= 2,
 *       SPC Lambda >= 4; a single leaf is a frozen or information leaf.
 *   R7  Every multi-element sum runs in halving order
 *       v[i] += v[i + h], h = Lambda/2 ... 1; ties in |alpha| go to the lower
 *       index.
 *   R8  SPC candidates: the 8 flip patterns of the four least reliable
 *       positions with parity equal to the node's hard-decision parity, in
 *       ascending 4-bit mask order; PM delta = sum of the flipped |alpha|.
 *   R9  REP: the better candidate is HD(sum alpha) repeated, the other one
 *       costs that plus |sum alpha|.
 *   R10 The visit counter is kept per branching node (indexed by its first
 *       leaf, the path length at which the path branches); once L paths have
 *       branched there, stacked paths of length <= that leaf are deleted.
 *   R11 Stack order: a beats b iff pm(a) < pm(b), or equal pm and a is newer.
 *       Candidates of one expansion are inserted in candidate order and get
 *       sequence numbers in reverse order (candidate 0 is the newest).  A
 *       full stack takes a candidate only if its pm is strictly below the
 *       worst entry's, which it replaces.  The path being extended does not
 *       occupy a stack slot.
 *   R12 A complete path is pushed like any candidate.  When popped it is
 *       returned if there is no CRC or the CRC passes; after L CRC failures
 *       (or an empty stack) the first complete path popped is returned with
 *       status CRC_FAIL.
 *   R13 Construction by Bhattacharyya parameters with z0 = exp(-R * 10^(dB/10)).
 *   R14 CRC: init 0, no reflection, no final xor, MSB first over the message
 *       bits in increasing info-index order; the CRC occupies the last crc
 *       info positions.
 * Systematic encoding (Sec. 2.2.2, Sec. 4): the codeword itself carries the
 * K information bits on the information set A, x_A = info, with u frozen = 0
 * and x = u F^{(x)n}; the decoder then reads the message straight from the
 * final beta array instead of re-encoding it.
 * Optional scaled min-sum (not in the paper; the learnable form of the
 * genie-aided gradient below): every f output written at stage lambda is
 * multiplied by scales[lambda] in float32.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_CRC_FAIL 1
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)

/* schedule operations (Fig. fsscsch): alpha, beta and the node decoders */
enum {
    OR_ALPHA = 0, /* compute alpha of node (lambda, phi) from its parent */
    OR_BETA = 1,  /* combine odd node (lambda, phi) with its left sibling */
    OR_R0 = 2,
    OR_R1 = 3,
    OR_REP = 4,
    OR_SPC = 5,
    OR_LEAF0 = 6, /* frozen leaf */
    OR_LEAF1 = 7, /* information leaf */
    OR_INTERNAL = 8
};

typedef struct {
    int type, lam, phi;
} or_op;

static int is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

static int ilog2(int x) {
    int n = 0;
    while ((1 << n) < x) n++;
    return n;
}

/* ------------------------------------------------------------------------ */
/* Code construction (reading R13; the paper itself uses the 5G sequence,   */
/* Sec. 5).  Bhattacharyya parameters in the natural-order decoding tree: a */
/* left (f) child gets 2z - z^2, a right (g) child gets z^2.  Computed in   */
/* the log domain in double precision.                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    double lz;
    int idx;
} or_rel;

static int rel_cmp(const void *pa, const void *pb) {
    const or_rel *a = (const or_rel *)pa, *b = (const or_rel *)pb;
    if (a->lz < b->lz) return -1;
    if (a->lz > b->lz) return 1;
    /* equal parameter: the higher index is taken as more reliable */
    return (a->idx > b->idx) ? -1 : (a->idx < b->idx) ? 1 : 0;
}

int or_construct(int N, int K, double design_snr_db, uint8_t *frozen) {
    if (!is_pow2(N) || N < 2 || N > (1 << 15) || K < 1 || K > N || !frozen) return OR_EINVAL;
    double *lz = (double *)malloc(sizeof(double) * N);
    or_rel *r = (or_rel *)malloc(sizeof(or_rel) * N);
    if (!lz || !r) {
        free(lz);
        free(r);
        return OR_ENOMEM;
    }
    double R = (double)K / (double)N;
    lz[0] = -R * pow(10.0, design_snr_db / 10.0); /* ln z0 */
    for (int Lam = N; Lam >= 2; Lam /= 2) {
        for (int s = 0; s < N; s += Lam) {
            double v = lz[s];
            /* ln(2z - z^2) = ln z + ln(2 - z) = ln z + ln 2 + ln(1 - z/2) */
            lz[s] = v + log(2.0) + log1p(-0.5 * exp(v));
            lz[s + Lam / 2] = 2.0 * v;
        }
    }
    for (int i = 0; i < N; i++) {
        r[i].lz = lz[i];
        r[i].idx = i;
    }
    qsort(r, N, sizeof(or_rel), rel_cmp);
    for (int i = 0; i < N; i++) frozen[i] = 1;
    for (int k = 0; k < K; k++) frozen[r[k].idx] = 0;
    free(lz);
    free(r);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Encoding c = u F^{(x)n} as the n-stage XOR tree of Fig. encoder: at the  */
/* stage with branch size Lambda, x[s+i] ^= x[s+i+Lambda].                  */
/* ------------------------------------------------------------------------ */
void or_encode(const uint8_t *u, int N, uint8_t *x) {
    for (int i = 0; i < N; i++) x[i] = u[i] & 1;
    for (int Lam = 1; Lam < N; Lam *= 2)
        for (int s = 0; s < N; s += 2 * Lam)
            for (int i = 0; i < Lam; i++) x[s + i] ^= x[s + i + Lam];
}

/* CRC register after long division of the bit string (reading R14). */
static uint32_t crc_poly(int crc_len) {
    switch (crc_len) {
    case 8: return 0x07u;
    case 16: return 0x1021u;
    case 24: return 0xB2B117u; /* CRC-24C of Sec. 5 */
    default: return 0u;
    }
}

uint32_t or_crc(const uint8_t *bits, int nbits, int crc_len) {
    uint32_t poly = crc_poly(crc_len), reg = 0u;
    uint32_t top = 1u << (crc_len - 1), mask = (crc_len == 32) ? 0xFFFFFFFFu : ((1u << crc_len) - 1u);
    for (int i = 0; i < nbits; i++) {
        uint32_t fb = ((reg & top) ? 1u : 0u) ^ (uint32_t)(bits[i] & 1);
        reg = (reg << 1) & mask;
        if (fb) reg ^= poly;
    }
    return reg;
}

/* Place message (+ CRC, MSB first) on the information set and encode. */
int or_encode_msg(const uint8_t *msg, int N, int K, const uint8_t *frozen, int crc, uint8_t *codeword) {
    if (!is_pow2(N) || K < 1 || K > N || crc < 0 || crc >= K || (crc && !crc_poly(crc))) return OR_EINVAL;
    int Kmsg = K - crc;
    uint8_t *info = (uint8_t *)malloc(K), *u = (uint8_t *)calloc(N, 1);
    if (!info || !u) {
        free(info);
        free(u);
        return OR_ENOMEM;
    }
    for (int j = 0; j < Kmsg; j++) info[j] = msg[j] & 1;
    if (crc) {
        uint32_t reg = or_crc(msg, Kmsg, crc);
        for (int j = 0; j < crc; j++) info[Kmsg + j] = (reg >> (crc - 1 - j)) & 1u;
    }
    int k = 0, nf = 0;
    for (int i = 0; i < N; i++) {
        if (frozen[i]) {
            nf++;
            continue;
        }
        if (k < K) u[i] = info[k];
        k++;
    }
    free(info);
    if (nf != N - K) {
        free(u);
        return OR_EINVAL;
    }
    or_encode(u, N, codeword);
    free(u);
    return OR_OK;
}

/* Systematic encoding by its definition: find u with u_i = 0 off A and   */
/* (u F^{(x)n})_j = info_j on A.  F^{(x)n} has a 1 at (i, j) iff the bits  */
/* of j are a subset of those of i, so x_j = XOR of u_i over i containing  */
/* j: a unit triangular system, solved from the largest index of A down.  */
int or_encode_sys(const uint8_t *info, int N, const uint8_t *frozen, uint8_t *x) {
    if (!is_pow2(N)) return OR_EINVAL;
    uint8_t *u = (uint8_t *)calloc(N, 1);
    int *pos = (int *)malloc(sizeof(int) * N);
    if (!u || !pos) {
        free(u);
        free(pos);
        return OR_ENOMEM;
    }
    int K = 0;
    for (int i = 0; i < N; i++)
        if (!frozen[i]) pos[K++] = i;
    for (int k = K - 1; k >= 0; k--) {
        int j = pos[k];
        uint8_t acc = info[k] & 1;
        for (int t = k + 1; t < K; t++) {
            int i = pos[t];
            if ((i & j) == j) acc ^= u[i];
        }
        u[j] = acc;
    }
    or_encode(u, N, x);
    free(u);
    free(pos);
    return OR_OK;
}

/* message + CRC (as in or_encode_msg) placed systematically */
int or_encode_msg_sys(const uint8_t *msg, int N, int K, const uint8_t *frozen, int crc, uint8_t *codeword) {
    if (!is_pow2(N) || K < 1 || K > N || crc < 0 || crc >= K || (crc && !crc_poly(crc))) return OR_EINVAL;
    int nf = 0;
    for (int i = 0; i < N; i++) nf += frozen[i] ? 1 : 0;
    if (nf != N - K) return OR_EINVAL;
    int Kmsg = K - crc;
    uint8_t *info = (uint8_t *)malloc(K);
    if (!info) return OR_ENOMEM;
    for (int j = 0; j < Kmsg; j++) info[j] = msg[j] & 1;
    if (crc) {
        uint32_t reg = or_crc(msg, Kmsg, crc);
        for (int j = 0; j < crc; j++) info[Kmsg + j] = (reg >> (crc - 1 - j)) & 1u;
    }
    int rc = or_encode_sys(info, N, frozen, codeword);
    free(info);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Schedule (Sec. 3.1, Fig. fsscsch): built once per code by walking the    */
/* tree; a node is either decoded by its node operation or split into       */
/* alpha(left), <left>, alpha(right), <right>, beta(right).                 */
/* ------------------------------------------------------------------------ */
static int classify(const uint8_t *fr, int lam, int phi, int fast) {
    int Lam = 1 << lam, s = phi * Lam, nf = 0;
    if (lam == 0) return fr[s] ? OR_LEAF0 : OR_LEAF1;
    if (!fast) return OR_INTERNAL;
    for (int i = 0; i < Lam; i++) nf += fr[s + i] ? 1 : 0;
    if (nf == Lam) return OR_R0;
    if (nf == 0) return OR_R1;
    if (nf == Lam - 1 && !fr[s + Lam - 1]) return OR_REP;
    if (lam >= 2 && nf == 1 && fr[s]) return OR_SPC;
    return OR_INTERNAL;
}

static void build(const uint8_t *fr, int lam, int phi, int fast, or_op *ops, int *nops) {
    int t = classify(fr, lam, phi, fast);
    if (t != OR_INTERNAL) {
        ops[(*nops)++] = (or_op){t, lam, phi};
        return;
    }
    ops[(*nops)++] = (or_op){OR_ALPHA, lam - 1, 2 * phi};
    build(fr, lam - 1, 2 * phi, fast, ops, nops);
    ops[(*nops)++] = (or_op){OR_ALPHA, lam - 1, 2 * phi + 1};
    build(fr, lam - 1, 2 * phi + 1, fast, ops, nops);
    ops[(*nops)++] = (or_op){OR_BETA, lam - 1, 2 * phi + 1};
}

/* ops_out: 3 ints per op (type, lambda, phi).  Returns the op count. */
int or_schedule(int N, const uint8_t *frozen, int fast, int *ops_out, int max_ops) {
    if (!is_pow2(N) || N < 2 || N > (1 << 15)) return OR_EINVAL;
    or_op *ops = (or_op *)malloc(sizeof(or_op) * (4 * N));
    if (!ops) return OR_ENOMEM;
    int nops = 0;
    build(frozen, ilog2(N), 0, fast, ops, &nops);
    for (int t = 0; t < nops && t < max_ops; t++) {
        ops_out[3 * t] = ops[t].type;
        ops_out[3 * t + 1] = ops[t].lam;
        ops_out[3 * t + 2] = ops[t].phi;
    }
    free(ops);
    return nops;
}

/* ------------------------------------------------------------------------ */
/* Min-sum primitives, Eq. minsum with readings R1 and R2.                  */
/* ------------------------------------------------------------------------ */
static float f_op(float a, float b) {
    float aa = fabsf(a), ab = fabsf(b);
    float m = (aa < ab) ? aa : ab;
    return (signbit(a) != 0) != (signbit(b) != 0) ? -m : m;
}

static float g_op(float a, float b, int beta) { return beta ? b - a : b + a; }

static int hd(float x) { return x < 0.0f; }

/* halving-order sum of v[0..Lam) in place (reading R7) */
static float halving_sum(float *v, int Lam) {
    for (int h = Lam / 2; h >= 1; h /= 2)
        for (int i = 0; i < h; i++) v[i] = v[i] + v[i + h];
    return v[0];
}

/* ------------------------------------------------------------------------ */
/* Operation counting convention for the ALU roofline (shared by definition */
/* with the GPU counters, not by code):                                     */
/*   f or g element 2; node pass 2 per element (R-0/leaf 1 pass, REP 2,     */
/*   R-1 3, SPC 5); PM add 1 per candidate plus 1 per extra addend in its   */
/*   delta; beta combine 1 per 32-bit word; stack pop, insert attempt or    */
/*   prune 2*ceil(log2 D) (at least 2); beta restore N/32 words; CRC check  */
/*   crc*N/32; output re-encode n*N/32.  alpha recomputation is counted     */
/*   only when the popped path is not a child of the previous expansion.   */
/* ------------------------------------------------------------------------ */
static int words32(int N) { return N < 32 ? 1 : N / 32; }

typedef struct {
    int N, n, K, Kmsg, fast, D, L, crc;
    const uint8_t *frozen;
    or_op *ops;
    int nops;
    const float *llr;  /* stage n: channel LLRs */
    const float *scales; /* NULL, or per-stage factors on the f outputs (stage of the child) */
    float *amem;       /* stages 0..n-1; stage lambda has Lambda slots (Sec. 3.1) */
    float *alpha[17];
    uint8_t *beta;     /* in-place N-entry beta array (Sec. 4, Fig. fsscsbmem) */
    /* stack (Sec. 3.3): D-length arrays */
    int ns;
    float *pm;
    int *len, *sched, *expn;
    uint32_t *seq;
    uint8_t *valid, *bits;
    int *cnt;          /* visit counter per branching leaf start */
    uint32_t seq_next;
    int exp_next, last_exp;
    /* scratch */
    float *tmp;
    uint8_t *cand;     /* up to 8 candidate patterns of N bytes */
    uint8_t *xhat, *uhat, *first_bits;
    uint64_t st_iter, st_switch, st_ops, st_exp, st_maxcnt;
    int stack_cost;
    int systematic; /* message read from the codeword estimate (no re-encode) */
    /* optional trace for tests: per pop, the popped path's schedule position,
     * path metric and its beta array right after the restore */
    int trace_max, trace_n;
    int *trace_sched;
    float *trace_pm;
    uint8_t *trace_beta;
} or_dec;

static void dec_free(or_dec *d) {
    free(d->ops);
    free(d->amem);
    free(d->beta);
    free(d->pm);
    free(d->len);
    free(d->sched);
    free(d->expn);
    free(d->seq);
    free(d->valid);
    free(d->bits);
    free(d->cnt);
    free(d->tmp);
    free(d->cand);
    free(d->xhat);
    free(d->uhat);
    free(d->first_bits);
}

static int dec_init(or_dec *d, int N, int K, const uint8_t *frozen, int fast, int D, int L, int crc) {
    memset(d, 0, sizeof(*d));
    if (!is_pow2(N) || N < 2 || N > (1 << 15) || K < 1 || K > N || D < 1 || L < 1) return OR_EINVAL;
    if (crc < 0 || crc >= K || (crc && !crc_poly(crc))) return OR_EINVAL;
    int nf = 0;
    for (int i = 0; i < N; i++) nf += frozen[i] ? 1 : 0;
    if (nf != N - K) return OR_EINVAL;
    d->N = N;
    d->n = ilog2(N);
    d->K = K;
    d->Kmsg = K - crc;
    d->fast = fast;
    d->D = D;
    d->L = L;
    d->crc = crc;
    d->frozen = frozen;
    d->ops = (or_op *)malloc(sizeof(or_op) * 4 * N);
    d->amem = (float *)malloc(sizeof(float) * N);
    d->beta = (uint8_t *)calloc(N, 1);
    d->pm = (float *)malloc(sizeof(float) * D);
    d->len = (int *)malloc(sizeof(int) * D);
    d->sched = (int *)malloc(sizeof(int) * D);
    d->expn = (int *)malloc(sizeof(int) * D);
    d->seq = (uint32_t *)malloc(sizeof(uint32_t) * D);
    d->valid = (uint8_t *)calloc(D, 1);
    d->bits = (uint8_t *)calloc((size_t)D * N, 1);
    d->cnt = (int *)calloc(N + 1, sizeof(int));
    d->tmp = (float *)malloc(sizeof(float) * N);
    d->cand = (uint8_t *)malloc((size_t)8 * N);
    d->xhat = (uint8_t *)malloc(N);
    d->uhat = (uint8_t *)malloc(N);
    d->first_bits = (uint8_t *)malloc(N);
    if (!d->ops || !d->amem || !d->beta || !d->pm || !d->len || !d->sched || !d->expn || !d->seq || !d->valid ||
        !d->bits || !d->cnt || !d->tmp || !d->cand || !d->xhat || !d->uhat || !d->first_bits) {
        dec_free(d);
        return OR_ENOMEM;
    }
    build(frozen, d->n, 0, fast, d->ops, &d->nops);
    for (int lam = 0; lam < d->n; lam++) d->alpha[lam] = d->amem + (1 << lam) - 1;
    int lg = 0;
    while ((1 << lg) < D) lg++;
    d->stack_cost = 2 * (lg < 1 ? 1 : lg);
    return OR_OK;
}

static const float *alpha_stage(or_dec *d, int lam) { return lam == d->n ? d->llr : d->alpha[lam]; }

/* Eq. llrcalc for node (lambda, phi) from its parent at lambda + 1 */
static void calc_alpha(or_dec *d, int lam, int phi, int count) {
    int Lam = 1 << lam;
    const float *ap = alpha_stage(d, lam + 1);
    float *av = d->alpha[lam];
    if ((phi & 1) == 0) {
        if (d->scales) {
            const float sc = d->scales[lam];
            for (int i = 0; i < Lam; i++) av[i] = sc * f_op(ap[i], ap[i + Lam]);
        } else {
            for (int i = 0; i < Lam; i++) av[i] = f_op(ap[i], ap[i + Lam]);
        }
    } else {
        const uint8_t *bu = d->beta + (phi - 1) * Lam; /* beta of u = (lambda, phi - 1) */
        for (int i = 0; i < Lam; i++) av[i] = g_op(ap[i], ap[i + Lam], bu[i]);
    }
    if (count) d->st_ops += 2u * (uint64_t)Lam;
}

/* Alg. calp after a path switch: recompute the whole spine from the root */
static void calc_alpha_from_root(or_dec *d, int lam, int phi, int count) {
    if (lam == d->n) return;
    calc_alpha_from_root(d, lam + 1, phi >> 1, count);
    calc_alpha(d, lam, phi, count);
}

/* ---- stack (Sec. 2.2.5, Sec. 3.3) ---- */
static int beats(or_dec *d, int a, int b) {
    if (d->pm[a] < d->pm[b]) return 1;
    if (d->pm[a] > d->pm[b]) return 0;
    return d->seq[a] > d->seq[b];
}

static int stack_best(or_dec *d) {
    int best = -1;
    for (int j = 0; j < d->D; j++)
        if (d->valid[j] && (best < 0 || beats(d, j, best))) best = j;
    return best;
}

static int stack_worst(or_dec *d) {
    int worst = -1;
    for (int j = 0; j < d->D; j++)
        if (d->valid[j] && (worst < 0 || beats(d, worst, j))) worst = j;
    return worst;
}

/* insert one candidate whose full beta array is `bits` (reading R11) */
static void stack_insert(or_dec *d, float pm, int len, int sched, uint32_t seq, int expn, const uint8_t *bits) {
    int slot = -1;
    d->st_ops += (uint64_t)d->stack_cost;
    if (d->ns < d->D) {
        for (int j = 0; j < d->D; j++)
            if (!d->valid[j]) {
                slot = j;
                break;
            }
        d->ns++;
    } else {
        int w = stack_worst(d);
        if (!(pm < d->pm[w])) return; /* dropped */
        slot = w;
    }
    d->valid[slot] = 1;
    d->pm[slot] = pm;
    d->len[slot] = len;
    d->sched[slot] = sched;
    d->seq[slot] = seq;
    d->expn[slot] = expn;
    memcpy(d->bits + (size_t)slot * d->N, bits, d->N);
}

/* L-prune of Sec. 2.2.5 (reading R10) */
static void stack_prune(or_dec *d, int omega) {
    d->st_ops += (uint64_t)d->stack_cost;
    for (int j = 0; j < d->D; j++)
        if (d->valid[j] && d->len[j] <= omega) {
            d->valid[j] = 0;
            d->ns--;
        }
}

/* message bits of a codeword estimate: re-encode (F is an involution, Sec. */
/* 2.2.2) and read the information set in increasing index order; with    */
/* systematic encoding they are the codeword bits on the information set  */
static void extract_info(or_dec *d, const uint8_t *xhat, uint8_t *info /* K */) {
    const uint8_t *src = xhat;
    if (!d->systematic) {
        or_encode(xhat, d->N, d->uhat);
        src = d->uhat;
    }
    int k = 0;
    for (int i = 0; i < d->N; i++)
        if (!d->frozen[i]) info[k++] = src[i];
}

static int crc_passes(or_dec *d, const uint8_t *xhat) {
    uint8_t *info = d->cand; /* candidate buffer is free at this point */
    extract_info(d, xhat, info);
    uint32_t reg = or_crc(info, d->Kmsg, d->crc);
    for (int j = 0; j < d->crc; j++)
        if (info[d->Kmsg + j] != ((reg >> (d->crc - 1 - j)) & 1u)) return 0;
    return 1;
}

/* node decoders (Sec. 2.2.2, Sec. 2.2.4): fill candidate patterns and deltas */
typedef struct {
    int nc;
    float delta[8];
} or_cands;

/* two or four least reliable positions, ties to the lower index (R7) */
static void least_reliable(const float *a, int Lam, int k, int *m) {
    for (int j = 0; j < k; j++) {
        int best = -1;
        for (int i = 0; i < Lam; i++) {
            int used = 0;
            for (int q = 0; q < j; q++) used |= (m[q] == i);
            if (used) continue;
            if (best < 0 || fabsf(a[i]) < fabsf(a[best])) best = i;
        }
        m[j] = best;
    }
}

static float pen(or_dec *d, const float *a, const uint8_t *w, int Lam) {
    for (int i = 0; i < Lam; i++) d->tmp[i] = (w[i] != hd(a[i])) ? fabsf(a[i]) : 0.0f;
    return halving_sum(d->tmp, Lam);
}

static void node_candidates(or_dec *d, int type, int lam, or_cands *c) {
    int Lam = 1 << lam, N = d->N;
    const float *a = alpha_stage(d, lam);
    uint8_t *P = d->cand;
    switch (type) {
    case OR_LEAF1: {
        int h = hd(a[0]);
        P[0] = (uint8_t)h;
        c->delta[0] = 0.0f;
        P[N] = (uint8_t)(1 - h);
        c->delta[1] = fabsf(a[0]);
        c->nc = 2;
        d->st_ops += 2u + 2u;
        break;
    }
    case OR_REP: {
        for (int i = 0; i < Lam; i++) d->tmp[i] = a[i];
        float S = halving_sum(d->tmp, Lam);
        int b = hd(S);
        for (int i = 0; i < Lam; i++) {
            P[i] = (uint8_t)b;
            P[N + i] = (uint8_t)(1 - b);
        }
        float p0 = pen(d, a, P, Lam);
        c->delta[0] = p0;
        c->delta[1] = p0 + fabsf(S);
        c->nc = 2;
        d->st_ops += 4u * (uint64_t)Lam + 2u + 1u;
        break;
    }
    case OR_R1: {
        int m[2];
        least_reliable(a, Lam, 2, m);
        for (int k = 0; k < 4; k++) {
            for (int i = 0; i < Lam; i++) P[k * N + i] = (uint8_t)hd(a[i]);
        }
        P[1 * N + m[0]] ^= 1;
        P[2 * N + m[1]] ^= 1;
        P[3 * N + m[0]] ^= 1;
        P[3 * N + m[1]] ^= 1;
        c->delta[0] = 0.0f;
        c->delta[1] = fabsf(a[m[0]]);
        c->delta[2] = fabsf(a[m[1]]);
        c->delta[3] = fabsf(a[m[0]]) + fabsf(a[m[1]]);
        c->nc = 4;
        d->st_ops += 6u * (uint64_t)Lam + 4u + 1u;
        break;
    }
    case OR_SPC: {
        int m[4], q = 0, k = 0;
        for (int i = 0; i < Lam; i++) q ^= hd(a[i]);
        least_reliable(a, Lam, 4, m);
        for (int mask = 0; mask < 16; mask++) {
            int pc = __builtin_popcount((unsigned)mask);
            if ((pc & 1) != q) continue;
            float delta = 0.0f;
            for (int i = 0; i < Lam; i++) P[k * N + i] = (uint8_t)hd(a[i]);
            for (int j = 0; j < 4; j++)
                if (mask & (1 << j)) {
                    P[k * N + m[j]] ^= 1;
                    delta = delta + fabsf(a[m[j]]);
                }
            c->delta[k] = delta;
            d->st_ops += 1u + (uint64_t)(pc > 1 ? pc - 1 : 0);
            k++;
        }
        c->nc = k;
        d->st_ops += 10u * (uint64_t)Lam;
        break;
    }
    default: c->nc = 0;
    }
}

/* frozen leaf / Rate-0 node: beta = 0, PM += sum HD(alpha)|alpha| (Sec. 2.2.4) */
static float rate0(or_dec *d, int lam, int phi) {
    int Lam = 1 << lam;
    const float *a = alpha_stage(d, lam);
    for (int i = 0; i < Lam; i++) {
        d->beta[phi * Lam + i] = 0;
        d->tmp[i] = hd(a[i]) ? fabsf(a[i]) : 0.0f;
    }
    d->st_ops += 2u * (uint64_t)Lam + 1u;
    return halving_sum(d->tmp, Lam);
}

static void write_output(or_dec *d, const uint8_t *xhat, uint8_t *msg_out, uint8_t *cw_out) {
    uint8_t *info = d->cand;
    extract_info(d, xhat, info);
    if (msg_out) memcpy(msg_out, info, (size_t)d->Kmsg);
    if (cw_out) memcpy(cw_out, xhat, (size_t)d->N);
    if (!d->systematic) d->st_ops += (uint64_t)d->n * (uint64_t)words32(d->N);
}

/* FSSCS-RM search (Sec. 2.2.5, Sec. 3.3, Sec. 4) for one frame. */
static int scs_run(or_dec *d, const float *llr, uint8_t *msg_out, float *pm_out, uint8_t *cw_out) {
    int N = d->N;
    d->llr = llr;
    d->ns = 0;
    memset(d->valid, 0, (size_t)d->D);
    memset(d->cnt, 0, sizeof(int) * (size_t)(N + 1));
    d->st_iter = d->st_switch = d->st_ops = d->st_exp = d->st_maxcnt = 0;
    memset(d->beta, 0, (size_t)N);
    d->seq_next = 1;
    d->exp_next = 1;
    d->last_exp = 0;
    stack_insert(d, 0.0f, 0, 0, 0u, 0, d->beta); /* the initial path */
    int crc_fails = 0, have_first = 0;
    float first_pm = 0.0f;
    for (;;) {
        if (d->ns == 0) { /* every path deleted: reading R12 */
            if (have_first) {
                write_output(d, d->first_bits, msg_out, cw_out);
                *pm_out = first_pm;
            } else {
                if (msg_out) memset(msg_out, 0, (size_t)d->Kmsg);
                if (cw_out) memset(cw_out, 0, (size_t)N);
                *pm_out = INFINITY;
            }
            return OR_CRC_FAIL;
        }
        int j = stack_best(d);
        d->st_iter++;
        d->st_ops += (uint64_t)d->stack_cost;
        d->valid[j] = 0;
        d->ns--;
        float pm = d->pm[j];
        int sched = d->sched[j];
        int real_switch = (d->expn[j] != d->last_exp);
        /* restore the path's beta array (Sec. 4: no re-population needed) */
        memcpy(d->beta, d->bits + (size_t)j * N, (size_t)N);
        if (d->trace_n < d->trace_max) {
            d->trace_sched[d->trace_n] = sched;
            d->trace_pm[d->trace_n] = pm;
            memcpy(d->trace_beta + (size_t)d->trace_n * N, d->beta, (size_t)N);
            d->trace_n++;
        }
        if (real_switch) {
            d->st_switch++;
            d->st_ops += (uint64_t)words32(N);
        }
        if (sched == d->nops) { /* complete path */
            if (d->crc) d->st_ops += (uint64_t)d->crc * (uint64_t)words32(N);
            if (d->crc == 0 || crc_passes(d, d->beta)) {
                write_output(d, d->beta, msg_out, cw_out);
                *pm_out = pm;
                return OR_OK;
            }
            crc_fails++;
            if (!have_first) {
                have_first = 1;
                first_pm = pm;
                memcpy(d->first_bits, d->beta, (size_t)N);
            }
            if (crc_fails >= d->L) {
                write_output(d, d->first_bits, msg_out, cw_out);
                *pm_out = first_pm;
                return OR_CRC_FAIL;
            }
            continue;
        }
        /* walk the schedule up to the next branching node (Sec. 4) */
        int switched = 1; /* the oracle always recomputes alpha from the root */
        int t = sched;
        for (; t < d->nops; t++) {
            or_op op = d->ops[t];
            int Lam = 1 << op.lam;
            if (op.type == OR_ALPHA) {
                if (switched) {
                    calc_alpha_from_root(d, op.lam + 1, op.phi >> 1, real_switch);
                    switched = 0;
                }
                calc_alpha(d, op.lam, op.phi, 1);
            } else if (op.type == OR_BETA) {
                uint8_t *bl = d->beta + (op.phi - 1) * Lam, *br = d->beta + op.phi * Lam;
                for (int i = 0; i < Lam; i++) bl[i] ^= br[i];
                d->st_ops += (uint64_t)(Lam < 32 ? 1 : Lam / 32);
            } else if (op.type == OR_R0 || op.type == OR_LEAF0) {
                pm = pm + rate0(d, op.lam, op.phi);
            } else {
                break; /* branching node */
            }
        }
        int expn = d->exp_next++;
        d->last_exp = expn;
        d->st_exp++;
        if (t == d->nops) { /* reached the end: push the completed path */
            d->st_ops += 1u;
            stack_insert(d, pm, N, d->nops, d->seq_next++, expn, d->beta);
            continue;
        }
        or_op op = d->ops[t];
        int Lam = 1 << op.lam, s = op.phi * Lam;
        if (++d->cnt[s] >= d->L) stack_prune(d, s);
        if ((uint64_t)d->cnt[s] > d->st_maxcnt) d->st_maxcnt = (uint64_t)d->cnt[s];
        or_cands c;
        node_candidates(d, op.type, op.lam, &c);
        uint32_t base = d->seq_next;
        d->seq_next += (uint32_t)c.nc;
        for (int k = 0; k < c.nc; k++) {
            memcpy(d->beta + s, d->cand + (size_t)k * N, (size_t)Lam);
            stack_insert(d, pm + c.delta[k], s + Lam, t + 1, base + (uint32_t)(c.nc - 1 - k), expn, d->beta);
        }
    }
}

/* stats (optional, 5 entries): pops, path switches, counted ops, expansions,
 * largest number of paths that branched at one node */
int or_scs_decode_sx(const float *llr, int N, int K, const uint8_t *frozen, int fast, int D, int L, int crc,
                     const float *scales, int systematic, uint8_t *msg_out, float *pm_out, uint8_t *cw_out,
                     uint64_t *stats) {
    or_dec d;
    int rc = dec_init(&d, N, K, frozen, fast, D, L, crc);
    if (rc) return rc;
    d.scales = scales;
    d.systematic = systematic ? 1 : 0;
    float pm = 0.0f;
    rc = scs_run(&d, llr, msg_out, &pm, cw_out);
    if (pm_out) *pm_out = pm;
    if (stats) {
        stats[0] = d.st_iter;
        stats[1] = d.st_switch;
        stats[2] = d.st_ops;
        stats[3] = d.st_exp;
        stats[4] = d.st_maxcnt;
    }
    dec_free(&d);
    return rc;
}

/* or_scs_decode_sx with a trace of the first max_pops pops (test hook): for
 * pop k, sched_out[k] = the popped path's schedule position (the number of
 * schedule operations before it; nops for a complete path), pm_trace[k] its
 * path metric and beta_trace[k * N ...] its N-entry beta array after the
 * restore.  *n_traced = the pops recorded. */
int or_scs_decode_trace(const float *llr, int N, int K, const uint8_t *frozen, int fast, int D, int L, int crc,
                        int systematic, int max_pops, int *sched_out, float *pm_trace, uint8_t *beta_trace,
                        int *n_traced, uint8_t *msg_out, float *pm_out, uint8_t *cw_out, uint64_t *stats) {
    or_dec d;
    int rc = dec_init(&d, N, K, frozen, fast, D, L, crc);
    if (rc) return rc;
    d.systematic = systematic ? 1 : 0;
    d.trace_max = max_pops;
    d.trace_sched = sched_out;
    d.trace_pm = pm_trace;
    d.trace_beta = beta_trace;
    float pm = 0.0f;
    rc = scs_run(&d, llr, msg_out, &pm, cw_out);
    if (pm_out) *pm_out = pm;
    if (n_traced) *n_traced = d.trace_n;
    if (stats) {
        stats[0] = d.st_iter;
        stats[1] = d.st_switch;
        stats[2] = d.st_ops;
        stats[3] = d.st_exp;
        stats[4] = d.st_maxcnt;
    }
    dec_free(&d);
    return rc;
}

int or_scs_decode_s(const float *llr, int N, int K, const uint8_t *frozen, int fast, int D, int L, int crc,
                    const float *scales, uint8_t *msg_out, float *pm_out, uint8_t *cw_out, uint64_t *stats) {
    return or_scs_decode_sx(llr, N, K, frozen, fast, D, L, crc, scales, 0, msg_out, pm_out, cw_out, stats);
}

int or_scs_decode(const float *llr, int N, int K, const uint8_t *frozen, int fast, int D, int L, int crc,
                  uint8_t *msg_out, float *pm_out, uint8_t *cw_out, uint64_t *stats) {
    return or_scs_decode_s(llr, N, K, frozen, fast, D, L, crc, NULL, msg_out, pm_out, cw_out, stats);
}

/* B frames, row-major llr[B][N]; msg_out[B][K-crc]; stats_out[B][4] optional
 * (iterations, switches, counted ops, expansions) */
int or_scs_decode_batch_sx(const float *llr, int B, int N, int K, const uint8_t *frozen, int fast, int D, int L,
                           int crc, const float *scales, int systematic, uint8_t *msg_out, float *pm_out,
                           int8_t *status_out, uint64_t *stats_out) {
    or_dec d;
    int rc = dec_init(&d, N, K, frozen, fast, D, L, crc);
    if (rc) return rc;
    d.scales = scales;
    d.systematic = systematic ? 1 : 0;
    for (int b = 0; b < B; b++) {
        float pm = 0.0f;
        int st = scs_run(&d, llr + (size_t)b * N, msg_out ? msg_out + (size_t)b * (K - crc) : NULL, &pm, NULL);
        pm_out[b] = pm;
        status_out[b] = (int8_t)st;
        if (stats_out) {
            stats_out[4 * (size_t)b] = d.st_iter;
            stats_out[4 * (size_t)b + 1] = d.st_switch;
            stats_out[4 * (size_t)b + 2] = d.st_ops;
            stats_out[4 * (size_t)b + 3] = d.st_exp;
        }
    }
    dec_free(&d);
    return OR_OK;
}

int or_scs_decode_batch_s(const float *llr, int B, int N, int K, const uint8_t *frozen, int fast, int D, int L,
                          int crc, const float *scales, uint8_t *msg_out, float *pm_out, int8_t *status_out,
                          uint64_t *stats_out) {
    return or_scs_decode_batch_sx(llr, B, N, K, frozen, fast, D, L, crc, scales, 0, msg_out, pm_out, status_out,
                                  stats_out);
}

int or_scs_decode_batch(const float *llr, int B, int N, int K, const uint8_t *frozen, int fast, int D, int L, int crc,
                        uint8_t *msg_out, float *pm_out, int8_t *status_out, uint64_t *stats_out) {
    return or_scs_decode_batch_s(llr, B, N, K, frozen, fast, D, L, crc, NULL, msg_out, pm_out, status_out, stats_out);
}

/* ------------------------------------------------------------------------ */
/* Exact-f variant, bit-level (no fast nodes): the f of the box-plus rule   */
/* and the exact leaf metric ln(1 + exp(-(1 - 2u) alpha)); in double it     */
/* pins the search to maximum likelihood on tiny codes, in float it is the  */
/* reference of the GPU's exact-f decoder (decisions in the paper's FP32).  */
/* ------------------------------------------------------------------------ */
#define X(name) name##_f64
#define REAL double
#define LOG1P log1p
#define EXP exp
#define FABS fabs
#include "polar_oracle_exact.inc"
#undef X
#undef REAL
#undef LOG1P
#undef EXP
#undef FABS
#define X(name) name##_f32
#define REAL float
#define LOG1P log1pf
#define EXP expf
#define FABS fabsf
#include "polar_oracle_exact.inc"
#undef X
#undef REAL
#undef LOG1P
#undef EXP
#undef FABS

int or_scs_decode_exact(const double *llr, int N, int K, const uint8_t *frozen, int D, int L, uint8_t *cw_out,
                        double *pm_out) {
    return or_scs_decode_exact_f64(llr, N, K, frozen, D, L, cw_out, pm_out);
}

/* ------------------------------------------------------------------------ */
/* Genie-aided SC with per-stage min-sum scales (double precision).         */
/* alpha at every node is computed with the true partial sums: the f child  */
/* at stage lambda is scale[lambda] * f(a, b); g uses the transmitted bits.  */
/* Loss = mean over information leaves of softplus(-(1 - 2u_i) L_i).        */
/* Gradient by reverse accumulation through the tree.                       */
/* ------------------------------------------------------------------------ */
static double f_ms(double a, double b) {
    double m = fabs(a) < fabs(b) ? fabs(a) : fabs(b);
    return ((a < 0) != (b < 0)) ? -m : m;
}

/* tree[lambda][k], k in [0, N): all nodes of stage lambda side by side */
static void gsc_forward_tree(const double *llr, const uint8_t *x_stage /* (n+1) x N partial sums */, int N, int n,
                             const double *scale, double *tree /* (n+1) x N */) {
    for (int i = 0; i < N; i++) tree[(size_t)n * N + i] = llr[i];
    for (int lam = n - 1; lam >= 0; lam--) {
        int Lam = 1 << lam;
        const double *par = tree + (size_t)(lam + 1) * N;
        double *cur = tree + (size_t)lam * N;
        for (int ps = 0; ps < N; ps += 2 * Lam) {
            for (int i = 0; i < Lam; i++) {
                double a = par[ps + i], b = par[ps + i + Lam];
                cur[ps + i] = scale[lam] * f_ms(a, b);
                int beta = x_stage[(size_t)lam * N + ps + i]; /* true beta of the left child */
                cur[ps + Lam + i] = beta ? b - a : b + a;
            }
        }
    }
}

/* partial sums: x_stage[lambda][s..s+Lambda) = encoding of u[s..s+Lambda) */
static void partial_sums(const uint8_t *u, int N, int n, uint8_t *x_stage) {
    for (int lam = 0; lam <= n; lam++) {
        int Lam = 1 << lam;
        for (int s = 0; s < N; s += Lam) or_encode(u + s, Lam, x_stage + (size_t)lam * N + s);
    }
}

int or_gsc_forward(const double *llr, const uint8_t *u, int N, const double *scale, double *leaf_out) {
    if (!is_pow2(N) || N < 2) return OR_EINVAL;
    int n = ilog2(N);
    double *tree = (double *)malloc(sizeof(double) * (size_t)(n + 1) * N);
    uint8_t *xs = (uint8_t *)malloc((size_t)(n + 1) * N);
    if (!tree || !xs) {
        free(tree);
        free(xs);
        return OR_ENOMEM;
    }
    partial_sums(u, N, n, xs);
    gsc_forward_tree(llr, xs, N, n, scale, tree);
    memcpy(leaf_out, tree, sizeof(double) * N);
    free(tree);
    free(xs);
    return OR_OK;
}

/* B frames: loss (mean over frames and information leaves) and its gradient */
int or_gsc_loss_grad(const double *llr, const uint8_t *u, int B, int N, const uint8_t *frozen, const double *scale,
                     double *loss_out, double *grad_out /* n */) {
    if (!is_pow2(N) || N < 2 || B < 1) return OR_EINVAL;
    int n = ilog2(N), K = 0;
    for (int i = 0; i < N; i++) K += frozen[i] ? 0 : 1;
    if (K == 0) return OR_EINVAL;
    double *tree = (double *)malloc(sizeof(double) * (size_t)(n + 1) * N);
    double *adj = (double *)malloc(sizeof(double) * (size_t)(n + 1) * N);
    uint8_t *xs = (uint8_t *)malloc((size_t)(n + 1) * N);
    if (!tree || !adj || !xs) {
        free(tree);
        free(adj);
        free(xs);
        return OR_ENOMEM;
    }
    double loss = 0.0, norm = 1.0 / ((double)B * (double)K);
    for (int lam = 0; lam < n; lam++) grad_out[lam] = 0.0;
    for (int b = 0; b < B; b++) {
        const double *l = llr + (size_t)b * N;
        const uint8_t *ub = u + (size_t)b * N;
        partial_sums(ub, N, n, xs);
        gsc_forward_tree(l, xs, N, n, scale, tree);
        memset(adj, 0, sizeof(double) * (size_t)(n + 1) * N);
        for (int i = 0; i < N; i++) {
            if (frozen[i]) continue;
            double sgn = 1.0 - 2.0 * ub[i], z = -sgn * tree[i];
            loss += softplus_f64(z) * norm;
            /* d softplus(z)/dL = sigmoid(z) * (-sgn) */
            double sig = 1.0 / (1.0 + exp(-z));
            adj[i] = sig * (-sgn) * norm;
        }
        for (int lam = 0; lam < n; lam++) {
            int Lam = 1 << lam;
            const double *par = tree + (size_t)(lam + 1) * N;
            const double *cadj = adj + (size_t)lam * N;
            double *padj = adj + (size_t)(lam + 1) * N;
            for (int ps = 0; ps < N; ps += 2 * Lam) {
                for (int i = 0; i < Lam; i++) {
                    double a = par[ps + i], bb = par[ps + i + Lam];
                    double gl = cadj[ps + i], gr = cadj[ps + Lam + i];
                    /* left: scale * f(a, b) */
                    double fv = f_ms(a, bb);
                    grad_out[lam] += gl * fv;
                    double sa = a < 0 ? -1.0 : 1.0, sb = bb < 0 ? -1.0 : 1.0;
                    if (fabs(a) <= fabs(bb)) padj[ps + i] += gl * scale[lam] * sb;
                    else padj[ps + i + Lam] += gl * scale[lam] * sa;
                    /* right: b + (1 - 2 beta) a */
                    int beta = xs[(size_t)lam * N + ps + i];
                    padj[ps + i] += gr * (beta ? -1.0 : 1.0);
                    padj[ps + i + Lam] += gr;
                }
            }
        }
    }
    *loss_out = loss;
    free(tree);
    free(adj);
    free(xs);
    return OR_OK;
}
