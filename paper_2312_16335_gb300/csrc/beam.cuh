// Persistent best-first beam search over the primary vectors with a rerank over the
// secondary vectors (Sec. 2 "Search"; App. D: greedy traversal with backtracking,
// Vamana graph).  One warp serves one query at a time; warps pull queries from a
// global counter until the batch is exhausted.
//
// Per warp, shared memory holds the beam (scores + ids sorted best first, the top bit
// of an id marks "expanded"; merged in place), a visited cache, and the candidate
// buffers of one expansion.  The visited cache is a set-associative table that may forget ids
// (overwrite when a bucket is full) but never reports an unvisited id as visited;
// a forgotten id that is met again is rescored and then rejected by the merge,
// because it is either still in the beam (exact key match) or worse than the beam's
// last member (the last member only improves).  The beam is therefore identical to
// the one of an exact visited set.
//
// The cache holds either whole 32-bit ids (buckets of 4) or 16-bit tags (buckets of 8, twice
// the slots in the same bytes).  A tag names its id exactly: with 2^b buckets, id x is stored
// as the tag x >> b in bucket (x xor (x >> b)) mod 2^b, so the bucket and the tag give x back;
// tags run below 0xFFFF (the empty mark) while n <= 0xFFFF * 2^b.
#pragma once

#include "common.cuh"

namespace lv {

struct BeamParams {
    // primary store + graph
    const uint8_t *prim;
    int64_t prim_stride;
    int prim_chunks;  // 16-byte code chunks of a primary record
    int prim_dim;     // codes per record (build score)
    const int32_t *graph;
    int R;
    int64_t n;
    int32_t entry;
    // queries
    const float *qp;  // padded queries in the primary space (search mode)
    int ldq;
    const float *pmean;    // primary mean mu_B (prim_dim): cq = <q', mu_B>, sq = sum q' of each query
    const float *smean;    // secondary mean mu (D): cQ = <q, mu>, sQ = sum q (rerank), or NULL
    const int4 *desc;      // per query (k, L, r, max_hops) or NULL
    int4 uni;
    int64_t m;
    // secondary store (rerank)
    const uint8_t *sec;
    int64_t sec_stride;
    int sec_chunks;
    int sec_bits;  // 8: LVQ-8 records, 16: IEEE half vectors
    int metric;    // 0 inner product, 1 L2 score 2 <q, x> - ||x||^2
    const float *Q;  // unreduced queries m x D
    int D;
    // build mode
    const int32_t *qnodes;
    float mu2;
    // outputs
    int32_t *ids;
    float *scores;
    int ldo;
    int2 *stats;
    // rerank hand-off (RERANK): the best min(r, beam size) ids of query i go to
    // cand[i * ldc ..] and their count to cand_n[i]; cand_n[i] = -1 when r = 0 and the
    // query's results were written directly
    int32_t *cand;
    int *cand_n;
    int ldc;
    // scheduling / capacities
    int *work;
    int *status;
    int Lcap;   // beam capacity (multiple of 32)
    int Hcap;   // visited cache slots (power of two, >= 2 * Lcap)
    int hbits;  // log2(Hcap)
    int vbits;  // bits of a visited-cache slot: 32 (ids, buckets of 4) or 16 (tags, buckets of 8)
    int Rcap;   // candidate buffer capacity (multiple of 32, >= W * R)
    int W;      // search width: parents expanded per round (1..4, W * R <= 256)
    int T;      // warps per query (1, 2 or 4; divides W); Rcap = T * (W / T * R rounded up to 32)
    int warp_smem;  // shared bytes of one query (one team of T warps, or one half warp)
    int qpw;        // queries per warp: 1 (beam_kernel) or 2 (beam_half_kernel, beam_half.cuh)
    int64_t *slots;  // host side: when set, the search launchers report the query slots one
                     // launch keeps resident (blocks per SM x SMs x teams per block) and launch nothing
};

constexpr int WMAX = 4;
constexpr int CMAX = 256;  // candidates of one round (W * R)

// shared memory of one query: beam (8 Lcap), visited cache (Hcap slots of vbits / 8 bytes), 4
// candidate arrays (16 Rcap), the scorer's query (qbytes, a multiple of 16), control words (64)
inline int beam_warp_smem(int Lcap, int Hcap, int vbits, int Rcap, int qbytes) {
    return 8 * Lcap + vbits / 8 * Hcap + 16 * Rcap + qbytes + 64;  // + 16 control words
}
// every id below n has a 16-bit tag in a cache of hcap slots (hcap / 8 buckets of 8 tags)
inline bool tags_fit(int64_t n, int hcap) {
    int b = 0;
    while ((8 << b) < hcap) ++b;
    return hcap >= 64 && n >= 1 && ((n - 1) >> b) < 0xFFFF;
}
// candidate capacity of a team: T slices of W / T parents' neighbours, each rounded up to 32
inline int beam_rcap(int W, int T, int R) { return T * ((W / T * R + 31) / 32 * 32); }
// shared bytes of the LVQ scorer's query limbs (nc chunks per lane, see LvqIntScorer)
inline int lvq_query_bytes(int bits, int nc) { return bits == 32 ? 0 : 4 * nc * 3 * (bits == 8 ? 1 : 2) * 16; }

// Two queries per warp (beam_half.cuh).  Shared bytes of one query: beam (8 Lcap), visited cache
// of 16-bit tags (2 Hcap), candidate ids, scores and beam positions (12 Rcap), positions by rank
// (2 Rcap), the scorer's query
constexpr int HALF_IDS = 8;  // adjacency ids one lane gathers per round: width * R <= 16 * 8
inline int half_query_smem(int Lcap, int Hcap, int Rcap, int qbytes) {
    return 8 * Lcap + 2 * Hcap + 14 * Rcap + qbytes;
}
// candidate capacity: the round's width * R ids, rounded up to 16 (keeps the layout 16-byte aligned)
inline int half_rcap(int W, int R) { return (W * R + 15) / 16 * 16; }
// the 16-bit tags of a visited cache of hcap slots (hcap / 4 buckets) name every id below n
inline bool half_tags_fit(int64_t n, int hcap) {
    int b = 0;
    while ((4 << b) < hcap) ++b;
    return hcap >= 64 && n >= 1 && ((n - 1) >> b) < 0xFFFF;
}

// --------------------------------------------------------------------------------
// Primary scorer with an integer query: q' is held as 24-bit fixed point
// q_int = round(q' / scale), scale = max|q'| / (2^23 - 1), split into three byte limbs
// q_int = 2^16 h + 2^8 m + l (h signed, m and l unsigned), so that <q_int, codes> is three
// dp4a chains per 4 codes.  The quantisation error of q' is at most scale / 2 per entry,
// i.e. |error of delta * <q', codes>| <= 2^-24 * d * (max x - min x) * max|q'|, about
// 2e-5 * ||q'|| * ||x|| at d = 160 -- inside the float32 path's 1e-4 tolerance.
// 4 lanes per record, 8 records per pass (16 when enough candidates are pending).
// --------------------------------------------------------------------------------
__device__ __forceinline__ int dp4a_su(uint32_t s8x4, uint32_t u8x4, int c) {
    int d;
    asm("dp4a.s32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(s8x4), "r"(u8x4), "r"(c));
    return d;
}
__device__ __forceinline__ int dp4a_uu(uint32_t a, uint32_t b, int c) {
    int d;
    asm("dp4a.u32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// L2: the score is 2 x (decoded inner product) - ||x||^2, the norm read from the record's second
// constants chunk (chunk CH + 1)
template <int NC, int BITS, bool L2 = false>
struct LvqIntScorer {
    static constexpr int CPC = BITS == 8 ? 16 : 32;  // codes per 16-byte chunk
    static constexpr int V4 = BITS == 8 ? 1 : 2;     // 16-byte limb vectors per limb and chunk
    // The limbs live in the warp's shared memory, chunk c at lq[(3 c + limb) V4 ..], limb 0 = h,
    // 1 = m, 2 = l, for the 4 NC chunks a group of 4 lanes covers (chunks >= CH are zero).
    static constexpr int QBYTES = 4 * NC * 3 * V4 * 16;
    // the 128-byte lines holding a record's first and last byte are prefetched into L2 as soon as the
    // visited test admits its id, so that the scorer's passes after the first one find the record
    // there (all of it when it spans at most two lines, as the 192-byte records of d = 160 do)
    static constexpr bool PREFETCH = true;
    __device__ __forceinline__ int rec_bytes() const { return 16 * (CH + 1 + (L2 ? 1 : 0)); }
    const uint4 *lq;
    float cq, sq, scale;
    int CH;
    const uint8_t *base;
    int64_t stride;

    // every warp of the team computes the scale; the writer stores the limbs
    __device__ __forceinline__ void setup(const BeamParams &p, int64_t qi, int lane, void *qsmem, bool writer) {
        CH = p.prim_chunks;
        base = p.prim;
        stride = p.prim_stride;
        const float *row = p.qp + qi * p.ldq;
        // the per-query constants of the decoded inner product: cq = <q', mu_B>, sq = sum q'
        float amax = 0.f, c = 0.f, s = 0.f;
        for (int j = lane; j < CH * CPC; j += 32) {
            const float v = row[j];
            amax = fmaxf(amax, fabsf(v));
            if (j < p.prim_dim) {
                c = fmaf(v, p.pmean[j], c);
                s += v;
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            amax = fmaxf(amax, __shfl_xor_sync(FULL, amax, o));
            c += __shfl_xor_sync(FULL, c, o);
            s += __shfl_xor_sync(FULL, s, o);
        }
        cq = c;
        sq = s;
        scale = amax > 0.f ? amax / 8388607.0f : 1.0f;
        const float inv = amax > 0.f ? 8388607.0f / amax : 0.f;
        uint32_t *dst = reinterpret_cast<uint32_t *>(qsmem);
        for (int c = lane; writer && c < 4 * NC; c += 32) {
#pragma unroll
            for (int w = 0; w < 4 * V4; ++w) {
                uint32_t h = 0, mm = 0, l = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    // element of this limb byte: LVQ-8 word w holds codes 4w..4w+3;
                    // LVQ-4 words 2i / 2i+1 hold the low / high nibbles of bytes 4i..4i+3
                    const int e = BITS == 8 ? 4 * w + b : 8 * (w >> 1) + 2 * b + (w & 1);
                    int qv = 0;
                    if (c < CH) {
                        qv = __float2int_rn(row[c * CPC + e] * inv);
                        qv = max(-8388607, min(8388607, qv));
                    }
                    h |= (uint32_t)((qv >> 16) & 0xff) << (8 * b);
                    mm |= (uint32_t)((qv >> 8) & 0xff) << (8 * b);
                    l |= (uint32_t)(qv & 0xff) << (8 * b);
                }
                dst[(3 * c + 0) * 4 * V4 + w] = h;
                dst[(3 * c + 1) * 4 * V4 + w] = mm;
                dst[(3 * c + 2) * 4 * V4 + w] = l;
            }
        }
        __syncwarp();
        lq = reinterpret_cast<const uint4 *>(qsmem);
    }

    template <int P>
    __device__ __forceinline__ void pass(const int *ids, float *out, int b, int cnt, int lane) const {
        const int g = lane & 3, grp = lane >> 2;
        const int holder = (lane & ~3) | (CH & 3);
        uint4 v[P][NC];
        int j[P];
#pragma unroll
        for (int r = 0; r < P; ++r) {
            j[r] = b + 8 * r + grp;
            const int id = j[r] < cnt ? ids[j[r]] : -1;
            const uint8_t *rec = base + (int64_t)(id < 0 ? 0 : id) * stride;
#pragma unroll
            for (int t = 0; t < NC; ++t) {
                const int c = g + 4 * t;
                v[r][t] = (c <= CH + (L2 ? 1 : 0) && id >= 0) ? ldg_stream(rec + 16 * c) : make_uint4(0, 0, 0, 0);
            }
        }
        int sh[P], sm[P], sl[P];
#pragma unroll
        for (int r = 0; r < P; ++r) sh[r] = sm[r] = sl[r] = 0;
#pragma unroll
        for (int t = 0; t < NC; ++t) {
            const uint4 *L4 = lq + (g + 4 * t) * 3 * V4;
#pragma unroll
            for (int vv = 0; vv < V4; ++vv) {
                const uint4 h4 = L4[vv], m4 = L4[V4 + vv], l4 = L4[2 * V4 + vv];
                const uint32_t hw[4] = {h4.x, h4.y, h4.z, h4.w};
                const uint32_t mw[4] = {m4.x, m4.y, m4.z, m4.w};
                const uint32_t lw[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
                for (int r = 0; r < P; ++r) {
                    const uint32_t w4[4] = {v[r][t].x, v[r][t].y, v[r][t].z, v[r][t].w};
                    if (BITS == 8) {
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            sh[r] = dp4a_su(hw[i], w4[i], sh[r]);
                            sm[r] = dp4a_uu(mw[i], w4[i], sm[r]);
                            sl[r] = dp4a_uu(lw[i], w4[i], sl[r]);
                        }
                    } else {
                        // limb words 4 vv .. 4 vv + 3 = low / high nibbles of code words 2 vv, 2 vv + 1
#pragma unroll
                        for (int i2 = 0; i2 < 2; ++i2) {
                            const uint32_t cw = w4[2 * vv + i2];
                            const uint32_t lo = cw & 0x0F0F0F0Fu, hi = (cw >> 4) & 0x0F0F0F0Fu;
                            sh[r] = dp4a_su(hw[2 * i2], lo, sh[r]);
                            sh[r] = dp4a_su(hw[2 * i2 + 1], hi, sh[r]);
                            sm[r] = dp4a_uu(mw[2 * i2], lo, sm[r]);
                            sm[r] = dp4a_uu(mw[2 * i2 + 1], hi, sm[r]);
                            sl[r] = dp4a_uu(lw[2 * i2], lo, sl[r]);
                            sl[r] = dp4a_uu(lw[2 * i2 + 1], hi, sl[r]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < P; ++r) {
            // partial sums of one lane are < 2^24 in magnitude: exact conversions
            float s = fmaf((float)sh[r], 65536.0f, fmaf((float)sm[r], 256.0f, (float)sl[r]));
            float dl = 0.f, lo = 0.f, x2 = 0.f;
#pragma unroll
            for (int t = 0; t < NC; ++t) {
                if (g + 4 * t == CH) {
                    dl = __uint_as_float(v[r][t].x);
                    lo = __uint_as_float(v[r][t].y);
                }
                if (L2 && g + 4 * t == CH + 1) x2 = __uint_as_float(v[r][t].y);
            }
            s += __shfl_xor_sync(FULL, s, 1);
            s += __shfl_xor_sync(FULL, s, 2);
            dl = __shfl_sync(FULL, dl, holder);
            lo = __shfl_sync(FULL, lo, holder);
            float sc = fmaf(dl * scale, s, fmaf(lo, sq, cq));
            if (L2) sc = fmaf(2.0f, sc, -__shfl_sync(FULL, x2, (lane & ~3) | ((CH + 1) & 3)));
            if (g == 0 && j[r] < cnt) out[j[r]] = sc;
        }
    }

    // scores of ids[0..cnt) into out[0..cnt) (shared memory); warp-collective
    __device__ __forceinline__ void score(const int *ids, float *out, int cnt, int lane) const {
        int b = 0;
        for (; b + 8 < cnt; b += 16) pass<2>(ids, out, b, cnt, lane);
        if (b < cnt) pass<1>(ids, out, b, cnt, lane);
    }
};

// --------------------------------------------------------------------------------
// Build scorer: the query is a database node's own primary record; the pair score is
// the exact build score (integer sums + a fixed float32 expression, see leanvec.h).
// --------------------------------------------------------------------------------
// sum of products of the unsigned codes held in two 16-byte chunks (exact)
template <int BITS>
__device__ __forceinline__ int code_dot(const uint4 &a, const uint4 &b) {
    unsigned s = 0u;
    if (BITS == 8) {
        s = __dp4a(a.x, b.x, s);
        s = __dp4a(a.y, b.y, s);
        s = __dp4a(a.z, b.z, s);
        s = __dp4a(a.w, b.w, s);
    } else {
        const uint32_t m = 0x0F0F0F0Fu;
        s = __dp4a(a.x & m, b.x & m, s);
        s = __dp4a((a.x >> 4) & m, (b.x >> 4) & m, s);
        s = __dp4a(a.y & m, b.y & m, s);
        s = __dp4a((a.y >> 4) & m, (b.y >> 4) & m, s);
        s = __dp4a(a.z & m, b.z & m, s);
        s = __dp4a((a.z >> 4) & m, (b.z >> 4) & m, s);
        s = __dp4a(a.w & m, b.w & m, s);
        s = __dp4a((a.w >> 4) & m, (b.w >> 4) & m, s);
    }
    return (int)s;
}

// L2: the pair score is -||y_a - y_b||^2 from the self scores N (second constants chunk)
template <int NC, int BITS, bool L2 = false>
struct BuildScorer {
    uint4 qc[NC];
    float qd, ql, qG, qH, qN, mu2, fdim;
    int CH;
    const uint8_t *base;
    int64_t stride;

    static constexpr int QBYTES = 0;
    static constexpr bool PREFETCH = false;
    __device__ __forceinline__ void setup(const BeamParams &p, int64_t qi, int lane, void *, bool) {
        CH = p.prim_chunks;
        base = p.prim;
        stride = p.prim_stride;
        mu2 = p.mu2;
        fdim = (float)p.prim_dim;
        const int g = lane & 3;
        const uint8_t *r = base + (int64_t)p.qnodes[qi] * stride;
#pragma unroll
        for (int t = 0; t < NC; ++t) {
            const int c = g + 4 * t;
            qc[t] = c < CH ? *reinterpret_cast<const uint4 *>(r + 16 * c) : make_uint4(0, 0, 0, 0);
        }
        float4 k = *reinterpret_cast<const float4 *>(r + 16 * CH);
        qd = k.x;
        ql = k.y;
        qG = k.z;
        qH = k.w;
        qN = L2 ? *reinterpret_cast<const float *>(r + 16 * CH + 16) : 0.f;
    }

    __device__ __forceinline__ void score(const int *ids, float *out, int cnt, int lane) const {
        const int g = lane & 3, grp = lane >> 2;
        const int holder = (lane & ~3) | (CH & 3);
        for (int b = 0; b < cnt; b += 16) {
            const int j0 = b + grp, j1 = b + 8 + grp;
            const int id0 = j0 < cnt ? ids[j0] : -1;
            const int id1 = j1 < cnt ? ids[j1] : -1;
            const uint8_t *r0 = base + (int64_t)(id0 < 0 ? 0 : id0) * stride;
            const uint8_t *r1 = base + (int64_t)(id1 < 0 ? 0 : id1) * stride;
            uint4 v0[NC], v1[NC];
#pragma unroll
            for (int t = 0; t < NC; ++t) {
                const int c = g + 4 * t;
                v0[t] = (c <= CH + (L2 ? 1 : 0) && id0 >= 0) ? ldg_stream(r0 + 16 * c) : make_uint4(0, 0, 0, 0);
                v1[t] = (c <= CH + (L2 ? 1 : 0) && id1 >= 0) ? ldg_stream(r1 + 16 * c) : make_uint4(0, 0, 0, 0);
            }
            int P0 = 0, P1 = 0;
            float4 k0 = make_float4(0, 0, 0, 0), k1 = make_float4(0, 0, 0, 0);
            float n0 = 0.f, n1 = 0.f;
#pragma unroll
            for (int t = 0; t < NC; ++t) {
                P0 += code_dot<BITS>(v0[t], qc[t]);
                P1 += code_dot<BITS>(v1[t], qc[t]);
                if (L2 && g + 4 * t == CH + 1) {
                    n0 = __uint_as_float(v0[t].x);
                    n1 = __uint_as_float(v1[t].x);
                }
                if (g + 4 * t == CH) {
                    k0 = make_float4(__uint_as_float(v0[t].x), __uint_as_float(v0[t].y), __uint_as_float(v0[t].z),
                                     __uint_as_float(v0[t].w));
                    k1 = make_float4(__uint_as_float(v1[t].x), __uint_as_float(v1[t].y), __uint_as_float(v1[t].z),
                                     __uint_as_float(v1[t].w));
                }
            }
            P0 += __shfl_xor_sync(FULL, P0, 1);
            P1 += __shfl_xor_sync(FULL, P1, 1);
            P0 += __shfl_xor_sync(FULL, P0, 2);
            P1 += __shfl_xor_sync(FULL, P1, 2);
            k0.x = __shfl_sync(FULL, k0.x, holder);
            k0.y = __shfl_sync(FULL, k0.y, holder);
            k0.z = __shfl_sync(FULL, k0.z, holder);
            k0.w = __shfl_sync(FULL, k0.w, holder);
            k1.x = __shfl_sync(FULL, k1.x, holder);
            k1.y = __shfl_sync(FULL, k1.y, holder);
            k1.z = __shfl_sync(FULL, k1.z, holder);
            k1.w = __shfl_sync(FULL, k1.w, holder);
            float s0 = build_pair_score(mu2, fdim, qd, ql, qG, qH, k0.x, k0.y, k0.z, k0.w, P0);
            float s1 = build_pair_score(mu2, fdim, qd, ql, qG, qH, k1.x, k1.y, k1.z, k1.w, P1);
            if (L2) {
                const int h2 = (lane & ~3) | ((CH + 1) & 3);
                s0 = l2_from_ip(s0, qN, __shfl_sync(FULL, n0, h2));
                s1 = l2_from_ip(s1, qN, __shfl_sync(FULL, n1, h2));
            }
            if (g == 0) {
                if (j0 < cnt) out[j0] = s0;
                if (j1 < cnt) out[j1] = s1;
            }
        }
    }
};

// Build scorer for long records (more code chunks than 4 lanes x 4 chunks hold, e.g. LVQ-8 codes of
// the unreduced vectors): a whole warp per record, lane l holds chunks l and l + 32 of the node's own
// record (CH + 1 <= 64); the same exact build score as BuildScorer.  4 records per pass.
template <int BITS, bool L2 = false>
struct BuildWarpScorer {
    static constexpr int QBYTES = 0;
    static constexpr bool PREFETCH = false;
    static constexpr int U = 4;
    uint4 qc[2];
    float qd, ql, qG, qH, qN, mu2, fdim;
    int CH;
    const uint8_t *base;
    int64_t stride;

    __device__ __forceinline__ void setup(const BeamParams &p, int64_t qi, int lane, void *, bool) {
        CH = p.prim_chunks;
        base = p.prim;
        stride = p.prim_stride;
        mu2 = p.mu2;
        fdim = (float)p.prim_dim;
        const uint8_t *r = base + (int64_t)p.qnodes[qi] * stride;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int c = lane + 32 * t;
            qc[t] = c < CH ? *reinterpret_cast<const uint4 *>(r + 16 * c) : make_uint4(0, 0, 0, 0);
        }
        const float4 k = *reinterpret_cast<const float4 *>(r + 16 * CH);
        qd = k.x;
        ql = k.y;
        qG = k.z;
        qH = k.w;
        qN = L2 ? *reinterpret_cast<const float *>(r + 16 * CH + 16) : 0.f;
    }

    __device__ __forceinline__ void score(const int *ids, float *out, int cnt, int lane) const {
        const int holder = CH & 31, tslot = CH >> 5;
        for (int b = 0; b < cnt; b += U) {
            uint4 v[U][2];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int id = b + u < cnt ? ids[b + u] : -1;
                const uint8_t *r = base + (int64_t)(id < 0 ? 0 : id) * stride;
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const int c = lane + 32 * t;
                    v[u][t] = (c <= CH + (L2 ? 1 : 0) && id >= 0) ? ldg_stream(r + 16 * c) : make_uint4(0, 0, 0, 0);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                // the query's chunks past CH are zero, so the constants chunk adds nothing
                int P = code_dot<BITS>(v[u][0], qc[0]) + code_dot<BITS>(v[u][1], qc[1]);
#pragma unroll
                for (int o = 16; o; o >>= 1) P += __shfl_xor_sync(FULL, P, o);
                const uint4 kv = tslot == 0 ? v[u][0] : v[u][1];
                const float kd = __shfl_sync(FULL, __uint_as_float(kv.x), holder);
                const float kl = __shfl_sync(FULL, __uint_as_float(kv.y), holder);
                const float kG = __shfl_sync(FULL, __uint_as_float(kv.z), holder);
                const float kH = __shfl_sync(FULL, __uint_as_float(kv.w), holder);
                float sc = build_pair_score(mu2, fdim, qd, ql, qG, qH, kd, kl, kG, kH, P);
                if (L2) {
                    const uint4 nv = ((CH + 1) >> 5) == 0 ? v[u][0] : v[u][1];
                    sc = l2_from_ip(sc, qN, __shfl_sync(FULL, __uint_as_float(nv.x), (CH + 1) & 31));
                }
                if (lane == 0 && b + u < cnt) out[b + u] = sc;
            }
        }
    }
};

// --------------------------------------------------------------------------------
// Whole-warp scorer for long records: float32 vectors (KIND 0, the full-dimensional
// baseline) or LVQ-8 secondary records (KIND 1, the rerank).  U records per pass.
// --------------------------------------------------------------------------------
// L2 (float32 records): 2 <q, x> - ||x||^2, the norm summed from the record itself
template <int NCW, int KIND, bool L2 = false>
struct WarpScorer {
    static constexpr int CPC = KIND == 0 ? 4 : 16;
    static constexpr int U = KIND == 0 ? (NCW > 4 ? 2 : 4) : 4;
    float q[NCW][CPC];
    float c0, s0;
    int CH;
    const uint8_t *base;
    int64_t stride;

    // qrow: qlen valid floats (the rest read as 0)
    __device__ __forceinline__ void setup_row(const float *qrow, int qlen, int chunks, const uint8_t *b,
                                              int64_t st, float cc, float ss, int lane) {
        CH = chunks;
        base = b;
        stride = st;
        c0 = cc;
        s0 = ss;
#pragma unroll
        for (int t = 0; t < NCW; ++t) {
            const int c = lane + 32 * t;
#pragma unroll
            for (int e = 0; e < CPC; ++e) {
                const int j = c * CPC + e;
                q[t][e] = (c < CH && j < qlen) ? qrow[j] : 0.0f;
            }
        }
    }

    static constexpr int QBYTES = 0;
    static constexpr bool PREFETCH = false;
    __device__ __forceinline__ void setup(const BeamParams &p, int64_t qi, int lane, void *, bool) {
        // full-dimensional float32 search: padded queries, no constants
        setup_row(p.qp + qi * p.ldq, p.ldq, p.prim_chunks, p.prim, p.prim_stride, 0.f, 0.f, lane);
    }

    __device__ __forceinline__ float dot1(const uint4 (&v)[NCW]) const {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, nn = 0.f;
#pragma unroll
        for (int t = 0; t < NCW; ++t) {
            if (KIND == 0) {
                a0 = fmaf(q[t][0], __uint_as_float(v[t].x), a0);
                a1 = fmaf(q[t][1], __uint_as_float(v[t].y), a1);
                a2 = fmaf(q[t][2], __uint_as_float(v[t].z), a2);
                a3 = fmaf(q[t][3], __uint_as_float(v[t].w), a3);
                if (L2) {
                    nn = fmaf(__uint_as_float(v[t].x), __uint_as_float(v[t].x), nn);
                    nn = fmaf(__uint_as_float(v[t].y), __uint_as_float(v[t].y), nn);
                    nn = fmaf(__uint_as_float(v[t].z), __uint_as_float(v[t].z), nn);
                    nn = fmaf(__uint_as_float(v[t].w), __uint_as_float(v[t].w), nn);
                }
            } else {
                const uint32_t w[4] = {v[t].x, v[t].y, v[t].z, v[t].w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    a0 = fmaf(q[t][4 * i + 0], byte_to_float<0>(w[i]), a0);
                    a1 = fmaf(q[t][4 * i + 1], byte_to_float<1>(w[i]), a1);
                    a2 = fmaf(q[t][4 * i + 2], byte_to_float<2>(w[i]), a2);
                    a3 = fmaf(q[t][4 * i + 3], byte_to_float<3>(w[i]), a3);
                }
            }
        }
        const float ip = (a0 + a1) + (a2 + a3);
        return L2 ? fmaf(2.0f, ip, -nn) : ip;  // per lane; the warp sum is the score
    }

    __device__ __forceinline__ void score(const int *ids, float *out, int cnt, int lane) const {
        const int tot = CH + (KIND == 1 ? 1 : 0);
        const int holder = CH & 31, tslot = CH >> 5;
        for (int b = 0; b < cnt; b += U) {
            uint4 v[U][NCW];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int id = b + u < cnt ? ids[b + u] : -1;
                const uint8_t *r = base + (int64_t)(id < 0 ? 0 : id) * stride;
#pragma unroll
                for (int t = 0; t < NCW; ++t) {
                    const int c = lane + 32 * t;
                    v[u][t] = (c < tot && id >= 0) ? ldg_stream(r + 16 * c) : make_uint4(0, 0, 0, 0);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                float s = dot1(v[u]);
#pragma unroll
                for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
                float dl = 0.f, lo = 0.f;
                if (KIND == 1) {
#pragma unroll
                    for (int t = 0; t < NCW; ++t)
                        if (t == tslot) {
                            dl = __uint_as_float(v[u][t].x);
                            lo = __uint_as_float(v[u][t].y);
                        }
                    dl = __shfl_sync(FULL, dl, holder);
                    lo = __shfl_sync(FULL, lo, holder);
                    s = fmaf(dl, s, fmaf(lo, s0, c0));
                }
                if (lane == 0 && b + u < cnt) out[b + u] = s;
            }
        }
    }
};

// team barrier: the T warps of one query (named barrier 1 + team; a warp barrier when T = 1)
__device__ __forceinline__ void team_sync(int T, int team) {
    if (T == 1)
        __syncwarp();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(1 + team), "r"(32 * T) : "memory");
}

// The top bit of each 16-bit half of w that is zero.  A borrow can also flag the upper half above
// a zero lower half: "some half is zero" is exact, and so is each flag when a zero lower half
// implies a zero upper one.
__device__ __forceinline__ unsigned zero_halves(unsigned w) { return (w - 0x00010001u) & ~w & 0x80008000u; }

// A bucket of 8 16-bit tags (empty = 0xFFFF; the empty slots are the bucket's last ones): true if
// `tag` is not in it, with the number of empty slots in `ne`
__device__ __forceinline__ bool bucket_tag_free(const uint4 v, unsigned tag, int &ne) {
    const unsigned tt = tag * 0x10001u;
    if (zero_halves(v.x ^ tt) | zero_halves(v.y ^ tt) | zero_halves(v.z ^ tt) | zero_halves(v.w ^ tt)) return false;
    ne = __popc(zero_halves(~v.x)) + __popc(zero_halves(~v.y)) + __popc(zero_halves(~v.z)) + __popc(zero_halves(~v.w));
    return true;
}

// --------------------------------------------------------------------------------
// The beam kernel.  A team of T = p.T warps serves one query: per round the W best
// unexpanded beam members are the parents, warp w of the team expands parents
// w, w + T, ... (stages their adjacency, tests the visited cache, scores the new ids and
// keeps those that can enter the beam), then warp 0 merges every warp's candidates into
// the beam.  The rounds are the same for every T, so are the results.
// BUILD: queries are nodes (p.qnodes), output = the final beam.
// RERANK: hand the top-r of the beam to the rerank kernel (rerank.cu).
// --------------------------------------------------------------------------------
// WT: the search width fixed at compile time (1 or 2; 0 = p.W, up to WMAX); TAGS: the visited
// cache holds 16-bit tags in buckets of 8 (p.vbits = 16) instead of ids in buckets of 4
template <class PS, bool BUILD, bool RERANK, int WT, bool TAGS = false>
__global__ void __launch_bounds__(256, 3) beam_kernel(const BeamParams p) {
    constexpr int WC = WT ? WT : WMAX;  // parents per round at most
    const int Wr = WT ? WT : p.W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int T = p.T, warp = threadIdx.x >> 5, team = warp / T, tw = warp - team * T;
    unsigned char *my = smem_raw + (size_t)team * p.warp_smem;
    float *const bS = reinterpret_cast<float *>(my);           // beam scores (sorted, best first)
    int *const bI = reinterpret_cast<int *>(bS + p.Lcap);      // beam ids, top bit = expanded
    int *const hash = bI + p.Lcap;                             // visited cache (ids or tags)
    uint16_t *const tags = reinterpret_cast<uint16_t *>(hash);
    int *const cI = hash + (TAGS ? p.Hcap / 2 : p.Hcap);      // ids of one expansion, then of
    float *const cS = reinterpret_cast<float *>(cI + p.Rcap);  // the candidates that enter (in place)
    int *const vPB = reinterpret_cast<int *>(cS + p.Rcap);     // beam members ahead of each (| rank << 16)
    int *const sPB = vPB + p.Rcap;                             // the same in candidate-rank order
    void *const qsm = sPB + p.Rcap;                            // the scorer's query
    int *const ctl = reinterpret_cast<int *>(reinterpret_cast<unsigned char *>(qsm) + PS::QBYTES);
    // ctl: [0] query, [1] size, [2] F, [4 + w] candidates of warp w, [8 + w] records scored by warp w
    // this warp's slice of the candidate arrays (Rw entries)
    const int Rw = p.Rcap / T;
    int *const wI = cI + tw * Rw;
    float *const wS = cS + tw * Rw;
    int *const wPB = vPB + tw * Rw;
    // visited cache: Hcap / 4 buckets of 4 ids or Hcap / 8 buckets of 8 tags, one 16-byte load
    // per lookup
    int4 *const hash4 = reinterpret_cast<int4 *>(hash);
    const int bshift = 34 - p.hbits;  // ids: 32 - log2(buckets)
    const int tb = p.hbits - 3;       // tags: log2(buckets)
    const unsigned tmask = (1u << tb) - 1u;
    const bool lead = tw == 0;
    PS ps;

    for (;;) {
        if (lead && lane == 0) ctl[0] = atomicAdd(p.work, 1);
        team_sync(T, team);
        const int64_t qi = ctl[0];
        if (qi >= p.m) break;
        int4 dq = p.desc ? p.desc[qi] : p.uni;
        int k = dq.x, L = dq.y, r = dq.z;
        const int mh = dq.w;
        if (L > p.Lcap || L < 1 || k > p.ldo || k < 0) {
            if (lead && lane == 0) atomicOr(p.status, ST_CAPACITY);
            L = min(max(L, 1), p.Lcap);
            k = min(max(k, 0), p.ldo);
        }
        r = min(max(r, 0), L);
        ps.setup(p, qi, lane, qsm, lead);
        for (int t = (tw * 32 + lane) * 4; t < (TAGS ? p.Hcap / 2 : p.Hcap); t += 128 * T)
            *reinterpret_cast<int4 *>(hash + t) = make_int4(-1, -1, -1, -1);  // empty: every bit set
        team_sync(T, team);
        const int entry = p.entry;
        if (lead) {
            if (lane == 0) {
                cI[0] = entry;
                if (TAGS) {
                    const unsigned tag = (unsigned)entry >> tb;
                    tags[8 * (((unsigned)entry ^ tag) & tmask)] = (uint16_t)tag;
                } else {
                    hash[4 * (int)(((unsigned)entry * 0x9E3779B1u) >> bshift)] = entry;
                }
            }
            __syncwarp();
            ps.score(cI, cS, 1, lane);
            __syncwarp();
            if (lane == 0) {
                bS[0] = cS[0];
                bI[0] = entry;
                ctl[1] = 1;
                ctl[2] = 0;
            }
        }
        team_sync(T, team);
        // every beam member before position F is expanded
        int size = 1, hops = 0, scored = lead ? 1 : 0, F = 0;
        const int maxh = mh > 0 ? mh : (int)(p.n < 0x7fffffff ? p.n : 0x7fffffff);

        while (hops < maxh) {
            // the W best unexpanded members of the beam: the first ones at positions >= F
            // (every warp of the team finds the same ones)
            int par[WC];
            int npar = 0;
            const int want = min(Wr, maxh - hops);
            for (int base = F & ~31; base < size && npar < want; base += 32) {
                const int i = base + lane;
                const bool un = i >= F && i < size && !(bI[i] & (int)EXPANDED);
                unsigned bal = __ballot_sync(FULL, un);
#pragma unroll
                for (int w = 0; w < WC; ++w) {
                    if (bal && npar < want && w == npar) {
                        par[w] = base + __ffs(bal) - 1;
                        bal &= bal - 1;
                        ++npar;
                    }
                }
            }
            if (npar == 0) break;
            F = par[0] + 1;
#pragma unroll
            for (int w = 1; w < WC; ++w)
                if (w < npar) F = par[w] + 1;
            hops += npar;

            // this warp's parents w = tw, tw + T, ...: neighbour ids staged in shared memory
            // (the slice's score buffer is free here), then tested against the visited cache
            // parent by parent (so an id shared by two parents of one warp is seen once)
            int *const stage = reinterpret_cast<int *>(wS);
            int nst = 0;
#pragma unroll
            for (int w = 0; w < WC; ++w) {
                if (w < npar && (w & (T - 1)) == tw) {  // T is a power of two
                    const int32_t *row = p.graph + (int64_t)(bI[par[w]] & ~(int)EXPANDED) * p.R;
                    for (int j = lane; j < p.R; j += 32) stage[nst + j] = __ldg(row + j);
                    nst += p.R;
                }
            }
            __syncwarp();
            int cnt = 0;
            for (int j0 = 0; j0 < nst; j0 += 64) {
                int u[2], slot[2];
                bool isnew[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = j0 + 32 * h + lane;
                    u[h] = j < nst ? stage[j] : -1;
                    if (u[h] >= p.n) { atomicOr(p.status, ST_CORRUPT); u[h] = -1; }
                }
                if constexpr (TAGS) {
                    // both halves' lookups first (one 16-byte load of 8 tags each), then the inserts:
                    // two new ids of one chunk that fall into one bucket take the same slot, and the
                    // one written last stays (the other may be scored again later)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        isnew[h] = false;
                        slot[h] = 0;
                        if (u[h] < 0) continue;
                        const unsigned x = (unsigned)u[h], tag = x >> tb;
                        const unsigned b = (x ^ tag) & tmask;
                        int ne = 0;
                        isnew[h] = bucket_tag_free(reinterpret_cast<const uint4 *>(hash4)[b], tag, ne);
                        // a bucket fills from its first slot and is overwritten only when full, so its
                        // empty slots are its last ne ones; when full, a hashed victim
                        slot[h] = 8 * (int)b + (ne ? 8 - ne : (int)((x * 0x85EBCA6Bu) >> 29));
                    }
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (isnew[h]) {
                            tags[slot[h]] = (uint16_t)((unsigned)u[h] >> tb);
                            if constexpr (PS::PREFETCH) {
                                const uint8_t *rec = ps.base + (int64_t)u[h] * ps.stride;
                                asm volatile("prefetch.global.L2 [%0];" ::"l"(rec));
                                asm volatile("prefetch.global.L2 [%0];" ::"l"(rec + ps.rec_bytes() - 1));
                            }
                        }
                        const unsigned bal = __ballot_sync(FULL, isnew[h]);
                        if (isnew[h]) wI[cnt + __popc(bal & lt)] = u[h];
                        cnt += __popc(bal);
                    }
                    // keep the next chunk's lookups (another parent's row) after these inserts: the
                    // 16-bit tag stores and the 16-byte bucket loads have different types, which the
                    // compiler may otherwise reorder (a warp's shared-memory accesses run in order)
                    asm volatile("" ::: "memory");
                } else {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        isnew[h] = false;
                        slot[h] = 0;
                        if (u[h] >= 0) {
                            const unsigned hv = (unsigned)u[h] * 0x9E3779B1u;
                            const int b = (int)(hv >> bshift);
                            const int4 v = hash4[b];
                            const int x = u[h];
                            if (v.x != x && v.y != x && v.z != x && v.w != x) {
                                isnew[h] = true;
                                slot[h] = 4 * b + (v.x < 0 ? 0 : v.y < 0 ? 1 : v.z < 0 ? 2 : v.w < 0 ? 3 : (int)((hv >> (bshift - 2)) & 3u));
                            }
                        }
                    }
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (isnew[h]) {
                            hash[slot[h]] = u[h];
                            if constexpr (PS::PREFETCH) {
                                const uint8_t *rec = ps.base + (int64_t)u[h] * ps.stride;
                                asm volatile("prefetch.global.L2 [%0];" ::"l"(rec));
                                asm volatile("prefetch.global.L2 [%0];" ::"l"(rec + ps.rec_bytes() - 1));
                            }
                        }
                        const unsigned bal = __ballot_sync(FULL, isnew[h]);
                        if (isnew[h]) wI[cnt + __popc(bal & lt)] = u[h];
                        cnt += __popc(bal);
                    }
                }
            }
            __syncwarp();
            int cv = 0;
            if (cnt > 0) {
                ps.score(wI, wS, cnt, lane);
                scored += cnt;
                __syncwarp();
                // keep candidates that can enter the beam and are not already in it (the beam
                // does not change until the merge)
                const bool full = size >= L;
                float tS = 0.f;
                int tI = 0;
                if (full) {
                    tS = bS[L - 1];
                    tI = bI[L - 1] & ~(int)EXPANDED;
                }
                for (int j0 = 0; j0 < cnt; j0 += 32) {
                    const int j = j0 + lane;
                    bool valid = false;
                    float s = 0.f;
                    int id = 0, pb = 0;
                    if (j < cnt) {
                        s = wS[j];
                        id = wI[j];
                        valid = !full || key_better(s, id, tS, tI);
                        if (valid) {
                            int lo = 0, hi = size;
                            while (lo < hi) {
                                const int mid = (lo + hi) >> 1;
                                const float ms = bS[mid];
                                bool better = ms > s;
                                if (ms == s) better = (bI[mid] & ~(int)EXPANDED) < id;
                                if (better)
                                    lo = mid + 1;
                                else
                                    hi = mid;
                            }
                            pb = lo;
                            if (pb < size && (bI[pb] & ~(int)EXPANDED) == id) valid = false;
                        }
                    }
                    const unsigned bal = __ballot_sync(FULL, valid);
                    __syncwarp();  // the chunk is read before it is compacted in place
                    if (valid) {
                        const int o = cv + __popc(bal & lt);
                        wI[o] = id;
                        wS[o] = s;
                        wPB[o] = pb;
                    }
                    cv += __popc(bal);
                }
            }
            if (T > 1) {
                if (lane == 0) ctl[4 + tw] = cv;
                team_sync(T, team);
            }
            if (lead) {
                // the parents are expanded now (the move below carries the flag along)
                __syncwarp();
                if (lane == 0)
#pragma unroll
                    for (int w = 0; w < WC; ++w)
                        if (w < npar) bI[par[w]] |= (int)EXPANDED;
                // the other warps' candidates follow warp 0's (in place: a slice only moves left)
                for (int w = 1; w < T; ++w) {
                    const int cw = ctl[4 + w];
                    const int *sI = cI + w * Rw;
                    const float *sS = cS + w * Rw;
                    const int *sP = vPB + w * Rw;
                    for (int j0 = 0; j0 < cw; j0 += 32) {
                        const int j = j0 + lane;
                        int id = 0, pb = 0;
                        float s = 0.f;
                        if (j < cw) {
                            id = sI[j];
                            s = sS[j];
                            pb = sP[j];
                        }
                        __syncwarp();
                        if (j < cw) {
                            cI[cv + j] = id;
                            cS[cv + j] = s;
                            vPB[cv + j] = pb;
                        }
                        __syncwarp();
                    }
                    cv += cw;
                }
                __syncwarp();
                if (cv > 0) {
                    // an id can appear twice in one round when two parents share a neighbour
                    // that the visited cache did not catch (another warp's concurrent test, or a
                    // forgotten id): keep the first copy
                    bool anydup = false;
                    if (Wr > 1) {
                        if (cv <= 32) {
                            // lanes past cv hold distinct negative keys that match nothing
                            const int id = lane < cv ? cI[lane] : -2 - lane;
                            const bool dup = (__match_any_sync(FULL, id) & lt) != 0u;
                            if (dup) vPB[lane] = -1;
                            anydup = __any_sync(FULL, dup);
                        } else {
                            bool d = false;
                            for (int j = lane; j < cv; j += 32) {
                                const int id = cI[j];
                                bool dup = false;
                                for (int u = 0; u < j; ++u) dup |= cI[u] == id;
                                if (dup) {
                                    vPB[j] = -1;
                                    d = true;
                                }
                            }
                            anydup = __any_sync(FULL, d);
                        }
                        __syncwarp();
                    }
                    if (anydup) {
                        int cv2 = 0;
                        for (int j0 = 0; j0 < cv; j0 += 32) {
                            const int j = j0 + lane;
                            const bool keep = j < cv && vPB[j] >= 0;
                            float s = 0.f;
                            int id = 0, pb = 0;
                            if (keep) {
                                s = cS[j];
                                id = cI[j];
                                pb = vPB[j];
                            }
                            const unsigned bal = __ballot_sync(FULL, keep);
                            __syncwarp();
                            if (keep) {
                                const int o = cv2 + __popc(bal & lt);
                                cI[o] = id;
                                cS[o] = s;
                                vPB[o] = pb;
                            }
                            cv2 += __popc(bal);
                            __syncwarp();
                        }
                        cv = cv2;
                    }
                    // rank of each candidate among the candidates; sPB[rank] = beam members ahead
                    for (int j = lane; j < cv; j += 32) {
                        const float s = cS[j];
                        const int id = cI[j];
                        int rank = 0;
                        for (int u = 0; u < cv; ++u) rank += key_better(cS[u], cI[u], s, id) ? 1 : 0;
                        const int pb = vPB[j];
                        sPB[rank] = pb;
                        vPB[j] = pb | (rank << 16);
                    }
                    __syncwarp();
                    // move beam members (in place, last chunk first; a member only moves right)
                    const int first = sPB[0];
                    for (int base = (size - 1) & ~31; base >= (first & ~31); base -= 32) {
                        const int i = base + lane;
                        float s = 0.f;
                        int id = 0, np = L;
                        if (i >= first && i < size) {
                            s = bS[i];
                            id = bI[i];
                            int lo = 0, hi = cv;
                            while (lo < hi) {
                                const int mid = (lo + hi) >> 1;
                                if (sPB[mid] <= i)
                                    lo = mid + 1;
                                else
                                    hi = mid;
                            }
                            np = i + lo;
                        }
                        __syncwarp();
                        if (np < L) {
                            bS[np] = s;
                            bI[np] = id;
                        }
                        __syncwarp();
                    }
                    // place the candidates (unexpanded)
                    for (int j = lane; j < cv; j += 32) {
                        const int x = vPB[j];
                        const int np = (x & 0xffff) + (x >> 16);
                        if (np < L) {
                            bS[np] = cS[j];
                            bI[np] = cI[j];
                        }
                    }
                    size = min(L, size + cv);
                    F = min(F, first);
                }
                if (T > 1 && lane == 0) {
                    ctl[1] = size;
                    ctl[2] = F;
                }
            }
            team_sync(T, team);
            if (T > 1) {
                size = ctl[1];
                F = ctl[2];
            }
        }

        if (T > 1) {
            if (lane == 0) ctl[8 + tw] = scored;
            team_sync(T, team);
            if (lead)
                for (int w = 1; w < T; ++w) scored += ctl[8 + w];
        }
        if (!lead) continue;
        if (p.stats && lane == 0) p.stats[qi] = make_int2(hops, scored);
        int32_t *oid = p.ids + qi * p.ldo;
        float *osc = p.scores + qi * p.ldo;
        if (BUILD) {
            for (int t = lane; t < L; t += 32) {
                oid[t] = t < size ? (bI[t] & ~(int)EXPANDED) : -1;
                osc[t] = t < size ? bS[t] : -INFINITY;
            }
        } else {
            if (RERANK && r > 0 && p.cand) {
                // the rerank kernel scores these with the secondary store and writes the results
                const int nr = min(r, size);
                int32_t *cd = p.cand + qi * p.ldc;
                for (int t = lane; t < nr; t += 32) cd[t] = bI[t] & ~(int)EXPANDED;
                if (lane == 0) p.cand_n[qi] = nr;
                __syncwarp();
                continue;
            }
            if (RERANK && p.cand_n && lane == 0) p.cand_n[qi] = -1;
            const int nres = min(k, size);
            for (int t = lane; t < nres; t += 32) {
                oid[t] = bI[t] & ~(int)EXPANDED;
                osc[t] = bS[t];
            }
            for (int t = nres + lane; t < p.ldo; t += 32) {
                oid[t] = -1;
                osc[t] = -INFINITY;
            }
        }
        __syncwarp();
    }
}

// launchers (one per translation unit); grid = persistent (SMs x resident blocks)
int launch_search_lvq8(const BeamParams &p, int nc, int block, size_t smem, int num_sms, cudaStream_t st);
int launch_search_lvq4(const BeamParams &p, int nc, int block, size_t smem, int num_sms, cudaStream_t st);
int launch_search_fp32(const BeamParams &p, int ncw, int block, size_t smem, int num_sms, cudaStream_t st);
// the same with p.vbits = 16 (visited cache of 16-bit tags); the three above pass such calls on
int launch_search_lvq8_tags(const BeamParams &p, int nc, int block, size_t smem, int num_sms, cudaStream_t st);
int launch_search_lvq4_tags(const BeamParams &p, int nc, int block, size_t smem, int num_sms, cudaStream_t st);
int launch_search_fp32_tags(const BeamParams &p, int ncw, int block, size_t smem, int num_sms, cudaStream_t st);
// two queries per warp: LVQ-8 primaries with nc = 1..4 chunks per lane, LVQ-4 with 1..3
int launch_search_half8(const BeamParams &p, int nc, int block, size_t smem, int num_sms, cudaStream_t st);
int launch_search_half4(const BeamParams &p, int nc, int block, size_t smem, int num_sms, cudaStream_t st);
int launch_build_search(const BeamParams &p, int bits, int nc, int block, size_t smem, int num_sms,
                        cudaStream_t st);
// scores the candidates the RERANK beam kernel handed over (p.cand, p.cand_n) and writes p.ids / p.scores
int launch_rerank(const BeamParams &p, int num_sms, cudaStream_t st);

// The search's launch shape (api.cu): beam / visited-cache / candidate capacities, width, warps and
// queries per warp (p.Lcap .. p.qpw) from the index and the caller's parameters, the block size and
// the dynamic shared memory.  `who` prefixes the error messages.
int search_shape(const lv_index *idx, const lv_search_params *params, BeamParams &p, int *block, size_t *smem,
                 const char *who);
// launches the beam kernel that fits the index's stores and p.qpw
int launch_beam_search(const lv_index *idx, const BeamParams &p, int block, size_t smem, cudaStream_t st);

}  // namespace lv
