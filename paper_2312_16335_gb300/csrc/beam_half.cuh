// Best-first beam search with two queries per warp (Sec. 2 "Search"; App. D: greedy traversal
// with backtracking over the Vamana graph).  Lanes 0-15 serve one query and lanes 16-31 another
// (the two "halves"); both halves run the same instruction stream in lockstep, each on its own
// beam, visited cache and candidates, and every warp-wide vote or shuffle is split by half.
// The rounds, the beam and the results are those of beam_kernel (beam.cuh) with one warp per
// query: the same parents per round, the same candidates entering the beam, the same merge.
//
// What changes is the number of queries in flight.  A round is a chain of dependent global and
// shared-memory loads; with two queries per warp each load's latency is paid once for two
// queries, and the shared memory of a query shrinks so that 40 queries fit on an SM (24 with one
// query per warp):
//   * the visited cache holds 16-bit tags: for a cache of 4 * 2^b slots (2^b buckets of 4), an
//     id x is stored as its tag x >> b in bucket (x + h(x >> b)) mod 2^b, h a multiplicative
//     hash; (bucket, tag) gives x back, so a tag match is an exact id match (the cache may
//     forget ids, never invent them) as long as every tag is below 0xFFFF, the empty mark, i.e.
//     n <= 0xFFFF * 2^b;
//   * the candidates' beam positions by rank are 16-bit.
// LVQ primaries only (the integer-limb scorer), one warp per query team, width 1 or 2 with
// width * R <= 128.
#pragma once

#include "beam.cuh"

namespace lv {

// this half's 16 bits of a warp ballot
__device__ __forceinline__ unsigned half_bits(unsigned bal, int hoff) { return (bal >> hoff) & 0xFFFFu; }

// The integer-limb primary scorer of LvqIntScorer (same limbs, same arithmetic, same scores) for
// a half warp: 4 lanes per record, 4 records per half and per record slot of a pass, up to three
// slots in flight.
template <int NC, int BITS, bool L2 = false>
struct HalfLvqScorer {
    static constexpr int CPC = BITS == 8 ? 16 : 32;
    static constexpr int V4 = BITS == 8 ? 1 : 2;
    static constexpr int QBYTES = 4 * NC * 3 * V4 * 16;
    const uint4 *lq;
    float cq, sq, scale;
    int CH;
    const uint8_t *base;
    int64_t stride;

    __device__ __forceinline__ void bind(const BeamParams &p, const void *qsmem) {
        CH = p.prim_chunks;
        base = p.prim;
        stride = p.prim_stride;
        lq = reinterpret_cast<const uint4 *>(qsmem);
        cq = sq = 0.f;
        scale = 1.f;
    }

    // warp-collective; the halves with `fresh` set take their query qi: per-query constants
    // cq = <q', mu_B>, sq = sum q', the 24-bit scale, and the limbs written to qsmem.  The sums run
    // in LvqIntScorer's order (lane hl plays that scorer's lanes hl and hl + 16), so the constants,
    // and with them every score, are bit for bit those of one query per warp.
    __device__ __forceinline__ void setup(const BeamParams &p, int64_t qi, int hl, void *qsmem, bool fresh) {
        const float *row = p.qp + (fresh ? qi : 0) * p.ldq;
        float amax = 0.f, c = 0.f, s = 0.f, c1 = 0.f, s1 = 0.f;
        for (int j = hl; fresh && j < CH * CPC; j += 32) {
            const float v = row[j];
            amax = fmaxf(amax, fabsf(v));
            if (j < p.prim_dim) {
                c = fmaf(v, p.pmean[j], c);
                s += v;
            }
            if (j + 16 < CH * CPC) {
                const float v1 = row[j + 16];
                amax = fmaxf(amax, fabsf(v1));
                if (j + 16 < p.prim_dim) {
                    c1 = fmaf(v1, p.pmean[j + 16], c1);
                    s1 += v1;
                }
            }
        }
        c += c1;
        s += s1;
#pragma unroll
        for (int o = 8; o; o >>= 1) {
            amax = fmaxf(amax, __shfl_xor_sync(FULL, amax, o));
            c += __shfl_xor_sync(FULL, c, o);
            s += __shfl_xor_sync(FULL, s, o);
        }
        if (!fresh) return;
        cq = c;
        sq = s;
        scale = amax > 0.f ? amax / 8388607.0f : 1.0f;
        const float inv = amax > 0.f ? 8388607.0f / amax : 0.f;
        uint32_t *dst = reinterpret_cast<uint32_t *>(qsmem);
        for (int c2 = hl; c2 < 4 * NC; c2 += 16) {
#pragma unroll
            for (int w = 0; w < 4 * V4; ++w) {
                uint32_t h = 0, mm = 0, l = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int e = BITS == 8 ? 4 * w + b : 8 * (w >> 1) + 2 * b + (w & 1);
                    int qv = 0;
                    if (c2 < CH) {
                        qv = __float2int_rn(row[c2 * CPC + e] * inv);
                        qv = max(-8388607, min(8388607, qv));
                    }
                    h |= (uint32_t)((qv >> 16) & 0xff) << (8 * b);
                    mm |= (uint32_t)((qv >> 8) & 0xff) << (8 * b);
                    l |= (uint32_t)(qv & 0xff) << (8 * b);
                }
                dst[(3 * c2 + 0) * 4 * V4 + w] = h;
                dst[(3 * c2 + 1) * 4 * V4 + w] = mm;
                dst[(3 * c2 + 2) * 4 * V4 + w] = l;
            }
        }
    }

    template <int P>
    __device__ __forceinline__ void pass(const int *ids, float *out, int b, int cnt, int lane) const {
        const int g = lane & 3, grp = (lane & 15) >> 2;
        const int holder = (lane & ~3) | (CH & 3);
        uint4 v[P][NC];
        int j[P];
#pragma unroll
        for (int r = 0; r < P; ++r) {
            j[r] = b + 4 * r + grp;
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

    // scores of ids[0..cnt) into out[0..cnt) (this half's shared memory); warp-collective, each
    // half with its own ids, out and cnt (0 for a half with nothing to score)
    __device__ __forceinline__ void score(const int *ids, float *out, int cnt, int lane) const {
        int b = 0;
        for (; __any_sync(FULL, b + 8 < cnt); b += 12) pass<3>(ids, out, b, cnt, lane);
        if (__any_sync(FULL, b + 4 < cnt))
            pass<2>(ids, out, b, cnt, lane);
        else if (__any_sync(FULL, b < cnt))
            pass<1>(ids, out, b, cnt, lane);
    }
};

// WT: search width (1 or 2).  Block: any number of warps; p.warp_smem = shared bytes of one query.
template <int NC, int BITS, bool L2, int WT>
__global__ void __launch_bounds__(320, 2) beam_half_kernel(const BeamParams p) {
    static_assert(WT == 1 || WT == 2, "width 1 or 2");
    using PS = HalfLvqScorer<NC, BITS, L2>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int hh = lane >> 4, hl = lane & 15, hoff = lane & 16;
    const unsigned lth = (1u << hl) - 1u;  // lanes of this half below this one (half-bit order)
    unsigned char *my = smem_raw + (size_t)((threadIdx.x >> 5) * 2 + hh) * p.warp_smem;
    float *const bS = reinterpret_cast<float *>(my);            // beam scores (sorted, best first)
    int *const bI = reinterpret_cast<int *>(bS + p.Lcap);       // beam ids, top bit = expanded
    uint16_t *const hash = reinterpret_cast<uint16_t *>(bI + p.Lcap);  // visited cache (tags)
    int *const cI = reinterpret_cast<int *>(hash + p.Hcap);     // ids of one expansion, then of
    float *const cS = reinterpret_cast<float *>(cI + p.Rcap);  // the candidates that enter (in place)
    int *const vPB = reinterpret_cast<int *>(cS + p.Rcap);      // beam members ahead (| rank << 16)
    uint16_t *const sPB = reinterpret_cast<uint16_t *>(vPB + p.Rcap);  // the same in rank order
    void *const qsm = sPB + p.Rcap;                             // the scorer's query limbs
    const uint2 *const hash4 = reinterpret_cast<const uint2 *>(hash);  // a bucket = 4 tags
    const int bb = p.hbits - 2;                                 // log2(buckets)
    const unsigned bmask = (1u << bb) - 1u;
    const int entry = p.entry;
    PS ps;
    ps.bind(p, qsm);

    int64_t qi = 0;
    bool live = false, exhausted = false;
    int size = 0, F = 0, hops = 0, scored = 0, L = 1, k = 0, r = 0, maxh = 0;
    for (;;) {
        // a half without a query takes the next one
        const bool need = !live && !exhausted;
        int nq = 0;
        if (need && hl == 0) nq = atomicAdd(p.work, 1);
        nq = __shfl_sync(FULL, nq, hoff);
        bool fresh = false;
        if (need) {
            if (nq < p.m) {
                qi = nq;
                fresh = true;
            } else {
                exhausted = true;
            }
        }
        if (!__any_sync(FULL, live || fresh)) break;
        if (__any_sync(FULL, fresh)) {
            if (fresh) {
                const int4 dq = p.desc ? p.desc[qi] : p.uni;
                k = dq.x;
                L = dq.y;
                r = dq.z;
                if (L > p.Lcap || L < 1 || k > p.ldo || k < 0) {
                    if (hl == 0) atomicOr(p.status, ST_CAPACITY);
                    L = min(max(L, 1), p.Lcap);
                    k = min(max(k, 0), p.ldo);
                }
                r = min(max(r, 0), L);
                maxh = dq.w > 0 ? dq.w : (int)(p.n < 0x7fffffff ? p.n : 0x7fffffff);
                for (int t = hl * 8; t < p.Hcap; t += 128)
                    *reinterpret_cast<uint4 *>(hash + t) = make_uint4(~0u, ~0u, ~0u, ~0u);
            }
            ps.setup(p, qi, hl, qsm, fresh);
            __syncwarp();
            if (fresh && hl == 0) {
                cI[0] = entry;
                const unsigned tag = (unsigned)entry >> bb;
                const unsigned hv = tag * 0x9E3779B1u;
                hash[4 * (((unsigned)entry + (hv >> (32 - bb))) & bmask)] = (uint16_t)tag;
            }
            __syncwarp();
            ps.score(cI, cS, fresh ? 1 : 0, lane);
            __syncwarp();
            if (fresh) {
                if (hl == 0) {
                    bS[0] = cS[0];
                    bI[0] = entry;
                }
                size = 1;
                hops = 0;
                scored = 1;
                F = 0;
                live = true;
            }
            __syncwarp();
        }

        // the W best unexpanded members of the beam: the first ones at positions >= F
        int par[WT];
#pragma unroll
        for (int w = 0; w < WT; ++w) par[w] = 0;
        int npar = 0;
        const int want = live ? min(WT, maxh - hops) : 0;
        for (int base = F & ~31;; base += 32) {
            const bool go = npar < want && base < size;
            if (!__any_sync(FULL, go)) break;
            const int i = base + hl, i2 = i + 16;
            const bool un = go && i >= F && i < size && !(bI[i] & (int)EXPANDED);
            const bool un2 = go && i2 >= F && i2 < size && !(bI[i2] & (int)EXPANDED);
            unsigned bal = half_bits(__ballot_sync(FULL, un), hoff) | (half_bits(__ballot_sync(FULL, un2), hoff) << 16);
#pragma unroll
            for (int w = 0; w < WT; ++w) {
                if (bal && npar < want && w == npar) {
                    par[w] = base + __ffs(bal) - 1;
                    bal &= bal - 1;
                    ++npar;
                }
            }
        }
        const bool fin = live && npar == 0;  // this half's traversal has ended
        const bool act = live && npar > 0;
        if (act) {
            F = par[0] + 1;
#pragma unroll
            for (int w = 1; w < WT; ++w)
                if (w < npar) F = par[w] + 1;
            hops += npar;
        }

        // the parents' neighbour ids, HALF_IDS per lane (flat index hl + 16 t over the parents' rows)
        const int tot = act ? npar * p.R : 0;
        const int32_t *row0 = p.graph + (int64_t)(act ? (bI[par[0]] & ~(int)EXPANDED) : 0) * p.R;
        const int32_t *row1 = row0;
        if (WT > 1 && npar > 1) row1 = p.graph + (int64_t)(bI[par[WT - 1]] & ~(int)EXPANDED) * p.R;
        int u[HALF_IDS];
#pragma unroll
        for (int t = 0; t < HALF_IDS; ++t) {
            const int f = hl + 16 * t;
            u[t] = -1;
            if (f < tot) {
                const bool second = WT > 1 && f >= p.R;
                u[t] = __ldg((second ? row1 : row0) + (second ? f - p.R : f));
            }
        }
#pragma unroll
        for (int t = 0; t < HALF_IDS; ++t)
            if (u[t] >= p.n) {
                atomicOr(p.status, ST_CORRUPT);
                u[t] = -1;
            }

        // visited test in two steps of 4 ids per lane (a step's inserts are seen by the next)
        int cnt = 0;
#pragma unroll
        for (int s2 = 0; s2 < HALF_IDS / 4; ++s2) {
            bool isnew[4];
            int slot[4];
            unsigned tg[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int x = u[4 * s2 + e];
                isnew[e] = false;
                slot[e] = 0;
                tg[e] = 0;
                if (x >= 0) {
                    const unsigned tag = (unsigned)x >> bb;
                    const unsigned hv = tag * 0x9E3779B1u;
                    const unsigned b = ((unsigned)x + (hv >> (32 - bb))) & bmask;
                    const uint2 v = hash4[b];
                    const unsigned tt = tag | (tag << 16);
                    if (!(__vcmpeq2(v.x, tt) | __vcmpeq2(v.y, tt))) {
                        isnew[e] = true;
                        tg[e] = tag;
                        const unsigned e0 = __vcmpeq2(v.x, 0xFFFFFFFFu), e1 = __vcmpeq2(v.y, 0xFFFFFFFFu);
                        const int w = e0 ? ((e0 & 0xFFFFu) ? 0 : 1)
                                         : e1 ? ((e1 & 0xFFFFu) ? 2 : 3) : (int)((hv >> (30 - bb)) & 3u);
                        slot[e] = 4 * (int)b + w;
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (isnew[e]) hash[slot[e]] = (uint16_t)tg[e];
                const unsigned bal = half_bits(__ballot_sync(FULL, isnew[e]), hoff);
                if (isnew[e]) cI[cnt + __popc(bal & lth)] = u[4 * s2 + e];
                cnt += __popc(bal);
            }
        }
        __syncwarp();

        // score the new ids; keep those that can enter the beam and are not already in it
        ps.score(cI, cS, cnt, lane);
        scored += cnt;
        __syncwarp();
        const bool full = size >= L;
        float tS = 0.f;
        int tI = 0;
        if (act && full) {
            tS = bS[L - 1];
            tI = bI[L - 1] & ~(int)EXPANDED;
        }
        // beam position of each candidate (beam members ahead of it: a prefix of the sorted beam),
        // two candidates per lane searched side by side in the same fixed number of steps
        const int top = size > 0 ? 1 << (31 - __clz(size)) : 0;  // largest power of two <= size
        int cv = 0;
        for (int j0 = 0; __any_sync(FULL, j0 < cnt); j0 += 32) {
            int jj[2], id[2], pos[2];
            float sc[2];
            bool valid[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                jj[e] = j0 + hl + 16 * e;
                valid[e] = false;
                sc[e] = 0.f;
                id[e] = 0;
                pos[e] = 0;
                if (jj[e] < cnt) {
                    sc[e] = cS[jj[e]];
                    id[e] = cI[jj[e]];
                    valid[e] = !full || key_better(sc[e], id[e], tS, tI);
                }
            }
            if (valid[0] || valid[1]) {
                for (int step = top; step > 0; step >>= 1) {
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int t = pos[e] + step;
                        if (t <= size) {
                            const float ms = bS[t - 1];
                            bool better = ms > sc[e];
                            if (ms == sc[e]) better = (bI[t - 1] & ~(int)EXPANDED) < id[e];
                            if (better) pos[e] = t;
                        }
                    }
                }
#pragma unroll
                for (int e = 0; e < 2; ++e)
                    if (valid[e] && pos[e] < size && (bI[pos[e]] & ~(int)EXPANDED) == id[e]) valid[e] = false;
            }
            const unsigned bal0 = half_bits(__ballot_sync(FULL, valid[0]), hoff);
            const unsigned bal1 = half_bits(__ballot_sync(FULL, valid[1]), hoff);
            __syncwarp();  // the chunk is read before it is compacted in place
            if (valid[0]) {
                const int o = cv + __popc(bal0 & lth);
                cI[o] = id[0];
                cS[o] = sc[0];
                vPB[o] = pos[0];
            }
            cv += __popc(bal0);
            if (valid[1]) {
                const int o = cv + __popc(bal1 & lth);
                cI[o] = id[1];
                cS[o] = sc[1];
                vPB[o] = pos[1];
            }
            cv += __popc(bal1);
        }

        // merge: the parents are expanded now (the move below carries the flag along)
        if (act && hl == 0)
#pragma unroll
            for (int w = 0; w < WT; ++w)
                if (w < npar) bI[par[w]] |= (int)EXPANDED;
        __syncwarp();
        if (WT > 1) {
            // an id can come twice in one round (two parents share a neighbour the visited cache
            // forgot, or one step's lanes met it together): keep the first copy.  A half with at
            // most 16 candidates takes one match over the warp (keys carry the half).
            const bool small = cv <= 16;
            const unsigned key = small && hl < cv ? (unsigned)cI[hl] * 2u + (unsigned)hh : 0xFFFFFFFFu - (unsigned)lane;
            bool d = (__match_any_sync(FULL, key) & ((1u << lane) - 1u)) != 0u;
            if (d) vPB[hl] = -1;
            if (!small) {
                for (int j = hl; j < cv; j += 16) {
                    const int id = cI[j];
                    bool dup = false;
                    for (int u2 = 0; u2 < j; ++u2) dup |= cI[u2] == id;
                    if (dup) {
                        vPB[j] = -1;
                        d = true;
                    }
                }
            }
            const bool anydup = half_bits(__ballot_sync(FULL, d), hoff) != 0u;
            __syncwarp();
            if (__any_sync(FULL, anydup)) {
                const int cvx = anydup ? cv : 0;
                int cv2 = 0;
                for (int j0 = 0; __any_sync(FULL, j0 < cvx); j0 += 16) {
                    const int j = j0 + hl;
                    const bool keep = j < cvx && vPB[j] >= 0;
                    float s = 0.f;
                    int id = 0, pb = 0;
                    if (keep) {
                        s = cS[j];
                        id = cI[j];
                        pb = vPB[j];
                    }
                    const unsigned bal = half_bits(__ballot_sync(FULL, keep), hoff);
                    __syncwarp();
                    if (keep) {
                        const int o = cv2 + __popc(bal & lth);
                        cI[o] = id;
                        cS[o] = s;
                        vPB[o] = pb;
                    }
                    cv2 += __popc(bal);
                    __syncwarp();
                }
                if (anydup) cv = cv2;
            }
        }
        // rank of each candidate among the candidates (two per lane); sPB[rank] = beam members ahead
        for (int j = hl; j < cv; j += 32) {
            const bool two = j + 16 < cv;
            const float sa = cS[j], sb = two ? cS[j + 16] : 0.f;
            const int ia = cI[j], ib = two ? cI[j + 16] : 0;
            int ra = 0, rb = 0;
            for (int u2 = 0; u2 < cv; ++u2) {
                const float su = cS[u2];
                const int iu = cI[u2];
                ra += key_better(su, iu, sa, ia) ? 1 : 0;
                rb += key_better(su, iu, sb, ib) ? 1 : 0;
            }
            const int pa = vPB[j];
            sPB[ra] = (uint16_t)pa;
            vPB[j] = pa | (ra << 16);
            if (two) {
                const int pb2 = vPB[j + 16];
                sPB[rb] = (uint16_t)pb2;
                vPB[j + 16] = pb2 | (rb << 16);
            }
        }
        __syncwarp();
        // move beam members (in place, last chunk of 32 first; a member only moves right): a member
        // at i moves by the number of candidates with at most i members ahead (a search over sPB)
        const int first = cv > 0 ? (int)sPB[0] : 0;
        const int ctop = cv > 0 ? 1 << (31 - __clz(cv)) : 0;
        for (int base = (size - 1) & ~31;; base -= 32) {
            const bool go = cv > 0 && base >= (first & ~31);
            if (!__any_sync(FULL, go)) break;
            float ms[2];
            int mi[2], np[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                ms[e] = 0.f;
                mi[e] = 0;
                np[e] = L;
            }
            const int i0 = base + hl;
            if (go && i0 + 16 >= first && i0 < size) {
                int lo[2] = {0, 0};
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int i = i0 + 16 * e;
                    if (i >= first && i < size) {
                        ms[e] = bS[i];
                        mi[e] = bI[i];
                    }
                }
                for (int step = ctop; step > 0; step >>= 1) {
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int t = lo[e] + step;
                        if (t <= cv && (int)sPB[t - 1] <= i0 + 16 * e) lo[e] = t;
                    }
                }
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int i = i0 + 16 * e;
                    if (i >= first && i < size) np[e] = i + lo[e];
                }
            }
            __syncwarp();
#pragma unroll
            for (int e = 0; e < 2; ++e)
                if (np[e] < L) {
                    bS[np[e]] = ms[e];
                    bI[np[e]] = mi[e];
                }
            __syncwarp();
        }
        // place the candidates (unexpanded)
        for (int j = hl; j < cv; j += 16) {
            const int x = vPB[j];
            const int np = (x & 0xffff) + (x >> 16);
            if (np < L) {
                bS[np] = cS[j];
                bI[np] = cI[j];
            }
        }
        if (cv > 0) {
            size = min(L, size + cv);
            F = min(F, first);
        }
        __syncwarp();

        // a finished half writes its results (or hands its beam to the rerank)
        if (fin) {
            if (p.stats && hl == 0) p.stats[qi] = make_int2(hops, scored);
            if (r > 0 && p.cand) {
                const int nr = min(r, size);
                int32_t *cd = p.cand + qi * p.ldc;
                for (int t = hl; t < nr; t += 16) cd[t] = bI[t] & ~(int)EXPANDED;
                if (hl == 0) p.cand_n[qi] = nr;
            } else {
                if (p.cand_n && hl == 0) p.cand_n[qi] = -1;
                int32_t *oid = p.ids + qi * p.ldo;
                float *osc = p.scores + qi * p.ldo;
                const int nres = min(k, size);
                for (int t = hl; t < nres; t += 16) {
                    oid[t] = bI[t] & ~(int)EXPANDED;
                    osc[t] = bS[t];
                }
                for (int t = nres + hl; t < p.ldo; t += 16) {
                    oid[t] = -1;
                    osc[t] = -INFINITY;
                }
            }
            live = false;
        }
        __syncwarp();
    }
}

// persistent launch (resident blocks x SMs); p.slots: report the query slots instead
template <int NC, int BITS, bool L2, int WT>
static int half_go(const BeamParams &p, int block, size_t smem, int num_sms, cudaStream_t st) {
    auto k = beam_half_kernel<NC, BITS, L2, WT>;
    LV_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    LV_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    int per_sm = 0;
    LV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem));
    if (per_sm < 1) return fail(LV_ERR_CAPACITY, "search: beam/visited capacity does not fit in shared memory");
    const int per_block = block / 16;  // queries served at once by one block
    if (p.slots) {
        *p.slots = (int64_t)per_sm * num_sms * per_block;
        return LV_OK;
    }
    const int64_t want = (p.m + per_block - 1) / per_block;
    const int64_t grid = std::min<int64_t>((int64_t)per_sm * num_sms, want);
    k<<<(unsigned)std::max<int64_t>(grid, 1), block, smem, st>>>(p);
    LV_CHECK_LAUNCH("beam_half_kernel");
    return LV_OK;
}

template <int NC, int BITS>
static int half_go_nc(const BeamParams &p, int block, size_t smem, int num_sms, cudaStream_t st) {
    if (p.metric) return p.W == 1 ? half_go<NC, BITS, true, 1>(p, block, smem, num_sms, st)
                                  : half_go<NC, BITS, true, 2>(p, block, smem, num_sms, st);
    return p.W == 1 ? half_go<NC, BITS, false, 1>(p, block, smem, num_sms, st)
                    : half_go<NC, BITS, false, 2>(p, block, smem, num_sms, st);
}


}  // namespace lv
