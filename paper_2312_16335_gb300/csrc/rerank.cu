// Rerank kernel (Sec. 2 "Search": the final candidates of the primary search are rescored
// with the full-dimensional LVQ-8 secondary vectors against the unreduced query, and the
// best k are kept).  The beam kernel hands over the top-r ids of every query
// (BeamParams::cand); here one warp takes one query, scores its r records whole-warp
// (16-byte coalesced loads of every record) and writes the top k.
#include <cuda_fp16.h>

#include "beam.cuh"

namespace lv {

// --------------------------------------------------------------------------------
// Rerank scorer (whole warp per record): LVQ-8 secondary records scored against the
// unreduced query held as 24-bit fixed point in three byte limbs (same scheme and
// error bound as LvqIntScorer, with D in place of d).  Lane l holds code chunks l and
// l + 32 (D <= 1008); 4 records per pass.
// --------------------------------------------------------------------------------
template <bool L2 = false>
struct SecIntScorer {
    static constexpr int NCW = 2, U = 4;
    uint32_t qh[NCW][4], qm[NCW][4], ql[NCW][4];
    float c0, s0, scale;
    int CH;
    const uint8_t *base;
    int64_t stride;

    __device__ __forceinline__ void setup(const float *qrow, int D, int chunks, const uint8_t *b, int64_t st,
                                          float cc, float ss, int lane) {
        CH = chunks;
        base = b;
        stride = st;
        c0 = cc;
        s0 = ss;
        float amax = 0.f;
        for (int j = lane; j < D; j += 32) amax = fmaxf(amax, fabsf(qrow[j]));
#pragma unroll
        for (int o = 16; o; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(FULL, amax, o));
        scale = amax > 0.f ? amax / 8388607.0f : 1.0f;
        const float inv = amax > 0.f ? 8388607.0f / amax : 0.f;
#pragma unroll
        for (int t = 0; t < NCW; ++t) {
            const int c = lane + 32 * t;
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                uint32_t h = 0, mm = 0, l = 0;
#pragma unroll
                for (int bb = 0; bb < 4; ++bb) {
                    const int j = c * 16 + 4 * w + bb;
                    int qv = 0;
                    if (c < CH && j < D) {
                        qv = __float2int_rn(qrow[j] * inv);
                        qv = max(-8388607, min(8388607, qv));
                    }
                    h |= (uint32_t)((qv >> 16) & 0xff) << (8 * bb);
                    mm |= (uint32_t)((qv >> 8) & 0xff) << (8 * bb);
                    l |= (uint32_t)(qv & 0xff) << (8 * bb);
                }
                qh[t][w] = h;
                qm[t][w] = mm;
                ql[t][w] = l;
            }
        }
    }

    __device__ __forceinline__ void score(const int *ids, float *out, int cnt, int lane) const {
        const int tot = CH + 1 + (L2 ? 1 : 0);
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
                int sh = 0, sm = 0, sl = 0;
#pragma unroll
                for (int t = 0; t < NCW; ++t) {
                    const uint32_t w4[4] = {v[u][t].x, v[u][t].y, v[u][t].z, v[u][t].w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        sh = dp4a_su(qh[t][i], w4[i], sh);
                        sm = dp4a_uu(qm[t][i], w4[i], sm);
                        sl = dp4a_uu(ql[t][i], w4[i], sl);
                    }
                }
                float s = fmaf((float)sh, 65536.0f, fmaf((float)sm, 256.0f, (float)sl));
#pragma unroll
                for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
                float dl = 0.f, lo = 0.f;
#pragma unroll
                for (int t = 0; t < NCW; ++t)
                    if (t == tslot) {
                        dl = __uint_as_float(v[u][t].x);
                        lo = __uint_as_float(v[u][t].y);
                    }
                dl = __shfl_sync(FULL, dl, holder);
                lo = __shfl_sync(FULL, lo, holder);
                float sc = fmaf(dl * scale, s, fmaf(lo, s0, c0));
                if (L2) {  // the original vector's squared norm: second constants chunk
                    const uint4 nv = ((CH + 1) >> 5) == 0 ? v[u][0] : v[u][1];
                    sc = fmaf(2.0f, sc, -__shfl_sync(FULL, __uint_as_float(nv.y), (CH + 1) & 31));
                }
                if (lane == 0 && b + u < cnt) out[b + u] = sc;
            }
        }
    }
};

// The best k of (S[0..n), I[0..n)) by (score desc, id asc), k rounds of a warp argmax;
// selected entries are marked by id -1.  Writes oid/osc[0..min(k, n)).
__device__ __forceinline__ void warp_topk(float *S, int *I, int n, int k, int32_t *oid, float *osc, int lane) {
    for (int r = 0; r < k && r < n; ++r) {
        float bs = -INFINITY;
        int bi = 0x7fffffff, bt = -1;
        for (int t = lane; t < n; t += 32) {
            const int id = I[t];
            if (id >= 0 && (bt < 0 || key_better(S[t], id, bs, bi))) {
                bs = S[t];
                bi = id;
                bt = t;
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const float os = __shfl_xor_sync(FULL, bs, o);
            const int oi = __shfl_xor_sync(FULL, bi, o);
            const int ot = __shfl_xor_sync(FULL, bt, o);
            if (ot >= 0 && (bt < 0 || key_better(os, oi, bs, bi))) {
                bs = os;
                bi = oi;
                bt = ot;
            }
        }
        if (lane == 0) {
            oid[r] = bi;
            osc[r] = bs;
            I[bt] = -1;
        }
        __syncwarp();
    }
}

// Rerank scorer for FP16 secondary records (whole warp per record): the unreduced query in
// float32 registers, lane l holds half chunks l, l + 32, ... (8 halves each; D <= 32 NCW 8); the
// halves are widened exactly to float32 and accumulated in float32.  4 records per pass.
template <int NCW, bool L2 = false>
struct Fp16SecScorer {
    static constexpr int U = 4;
    float q[NCW][8];
    int CH;
    const uint8_t *base;
    int64_t stride;

    __device__ __forceinline__ void setup(const float *qrow, int D, int chunks, const uint8_t *b, int64_t st, float,
                                          float, int lane) {
        CH = chunks;
        base = b;
        stride = st;
#pragma unroll
        for (int t = 0; t < NCW; ++t) {
            const int c = lane + 32 * t;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int j = 8 * c + e;
                q[t][e] = (c < CH && j < D) ? qrow[j] : 0.f;
            }
        }
    }

    __device__ __forceinline__ void score(const int *ids, float *out, int cnt, int lane) const {
        for (int b = 0; b < cnt; b += U) {
            uint4 v[U][NCW];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int id = b + u < cnt ? ids[b + u] : -1;
                const uint8_t *r = base + (int64_t)(id < 0 ? 0 : id) * stride;
#pragma unroll
                for (int t = 0; t < NCW; ++t) {
                    const int c = lane + 32 * t;
                    v[u][t] = (c < CH && id >= 0) ? ldg_stream(r + 16 * c) : make_uint4(0, 0, 0, 0);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                float a0 = 0.f, a1 = 0.f, nn = 0.f;
#pragma unroll
                for (int t = 0; t < NCW; ++t) {
                    const uint32_t w[4] = {v[u][t].x, v[u][t].y, v[u][t].z, v[u][t].w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float2 x = __half22float2(*reinterpret_cast<const __half2 *>(&w[i]));
                        a0 = fmaf(q[t][2 * i], x.x, a0);
                        a1 = fmaf(q[t][2 * i + 1], x.y, a1);
                        if (L2) nn = fmaf(x.y, x.y, fmaf(x.x, x.x, nn));
                    }
                }
                float s = a0 + a1;
                if (L2) s = fmaf(2.0f, s, -nn);  // 2 <q, x16> - ||x16||^2, summed over the warp below
#pragma unroll
                for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
                if (lane == 0 && b + u < cnt) out[b + u] = s;
            }
        }
    }
};

struct RerankParams {
    const uint8_t *sec;
    int64_t sec_stride;
    int sec_chunks;
    const float *Q;  // unreduced queries m x D
    int D;
    const float *smean;    // secondary mean mu (D) or NULL: cQ = <q, mu>, sQ = sum q per query
    const int4 *desc;      // per query (k, L, r, max_hops) or NULL
    int4 uni;
    int64_t m;
    const int32_t *cand;  // m x ldc candidate ids
    const int *cand_n;    // per query: candidates, or -1 = results already written
    int ldc;
    int32_t *ids;
    float *scores;
    int ldo;
};

constexpr int RR_WARPS = 4;

template <class SS>
__global__ void __launch_bounds__(32 * RR_WARPS) rerank_kernel(const RerankParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float *const rS = reinterpret_cast<float *>(smem_raw) + (size_t)wid * 2 * p.ldc;
    int *const rI = reinterpret_cast<int *>(rS + p.ldc);
    for (int64_t qi = (int64_t)blockIdx.x * RR_WARPS + wid; qi < p.m; qi += (int64_t)gridDim.x * RR_WARPS) {
        const int nr = min(p.cand_n[qi], p.ldc);
        if (nr < 0) continue;
        int k = p.desc ? p.desc[qi].x : p.uni.x;
        k = min(max(k, 0), p.ldo);
        const int32_t *cd = p.cand + qi * p.ldc;
        for (int t = lane; t < nr; t += 32) rI[t] = cd[t];
        __syncwarp();
        SS sc;
        const float *q = p.Q + qi * p.D;
        float cQ = 0.f, sQ = 0.f;
        if (p.smean) {
            for (int j = lane; j < p.D; j += 32) {
                const float v = q[j];
                cQ = fmaf(v, p.smean[j], cQ);
                sQ += v;
            }
            for (int o = 16; o; o >>= 1) {
                cQ += __shfl_xor_sync(FULL, cQ, o);
                sQ += __shfl_xor_sync(FULL, sQ, o);
            }
        }
        sc.setup(q, p.D, p.sec_chunks, p.sec, p.sec_stride, cQ, sQ, lane);
        sc.score(rI, rS, nr, lane);
        __syncwarp();
        int32_t *oid = p.ids + qi * p.ldo;
        float *osc = p.scores + qi * p.ldo;
        warp_topk(rS, rI, nr, k, oid, osc, lane);
        for (int t = min(k, nr) + lane; t < p.ldo; t += 32) {
            oid[t] = -1;
            osc[t] = -INFINITY;
        }
        __syncwarp();
    }
}

template <class SS>
static int go_rerank(const RerankParams &p, int num_sms, cudaStream_t st) {
    const size_t smem = (size_t)RR_WARPS * 2 * sizeof(float) * p.ldc;
    if (smem > 48 * 1024)
        LV_CUDA(cudaFuncSetAttribute(rerank_kernel<SS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t want = (p.m + RR_WARPS - 1) / RR_WARPS;
    const int64_t grid = std::min<int64_t>(want, (int64_t)num_sms * 64);
    rerank_kernel<SS><<<(unsigned)std::max<int64_t>(grid, 1), 32 * RR_WARPS, smem, st>>>(p);
    LV_CHECK_LAUNCH("rerank_kernel");
    return LV_OK;
}

template <bool L2>
static int launch_rerank_m(const BeamParams &bp, const RerankParams &p, int num_sms, cudaStream_t st) {
    if (bp.sec_bits == 16) {
        switch ((p.sec_chunks + 31) / 32) {
            case 1: return go_rerank<Fp16SecScorer<1, L2>>(p, num_sms, st);
            case 2: return go_rerank<Fp16SecScorer<2, L2>>(p, num_sms, st);
            case 3: return go_rerank<Fp16SecScorer<3, L2>>(p, num_sms, st);
            case 4: return go_rerank<Fp16SecScorer<4, L2>>(p, num_sms, st);
            default: return fail(LV_ERR_ARG, "rerank: FP16 secondaries longer than 1024 dimensions");
        }
    }
    return go_rerank<SecIntScorer<L2>>(p, num_sms, st);
}

int launch_rerank(const BeamParams &bp, int num_sms, cudaStream_t st) {
    RerankParams p;
    p.sec = bp.sec;
    p.sec_stride = bp.sec_stride;
    p.sec_chunks = bp.sec_chunks;
    p.Q = bp.Q;
    p.D = bp.D;
    p.smean = bp.smean;
    p.desc = bp.desc;
    p.uni = bp.uni;
    p.m = bp.m;
    p.cand = bp.cand;
    p.cand_n = bp.cand_n;
    p.ldc = bp.ldc;
    p.ids = bp.ids;
    p.scores = bp.scores;
    p.ldo = bp.ldo;
    if (bp.metric) return launch_rerank_m<true>(bp, p, num_sms, st);
    return launch_rerank_m<false>(bp, p, num_sms, st);
}

}  // namespace lv
