// BF16 tensor-core GEMM on the 5th-generation tensor cores (tcgen05, sm_103a):
//   C[M x N] (float32) = A[M x K] * B[N x K]^T,  A and B bf16, K-major (K contiguous).
// Used for the dense contractions of the path: the query projection q -> A q and the
// database projection x -> B x (Eq. 1), and the second moments K = sum x x^T
// (Sec. 2.2 "Efficiency", as Xt * Xt^T with Xt = X^T in bf16).
//
// One CTA (4 warps) owns a 128 x BN output tile and a range of K (split-K):
//   warp 0, one thread : TMA producer, 4-stage ring of (A 128x64, B BNx64) bf16 tiles
//                        in 128-byte-swizzled shared memory, mbarrier transaction counts;
//   warp 1, one thread : issues tcgen05.mma (M = 128, N = BN, K = 16 per instruction)
//                        with the float32 accumulator in tensor memory; tcgen05.commit
//                        releases each stage and finally signals the epilogue;
//   all 4 warps        : epilogue, tcgen05.ld of their 32 TMEM lanes, float32 stores.
// Every mbarrier wait is bounded: on time-out the kernel records LV status TIMEOUT,
// skips its remaining work, waits (bounded) for its own copies and frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"

namespace lv {

constexpr int TC_BM = 128, TC_STAGES = 4;
constexpr long long TC_SPIN_LIMIT = 1ll << 22;  // try_wait may suspend: keeps a give-up within seconds

struct TcParams {
    int M, N, K;
    int BN;
    int kb_per_split;
    float *C;        // direct output (split == 1) ...
    int ldc;
    float *partial;  // ... or partial[split][M][N] (split > 1)
    const float *row_scale;  // fp8: C[r][c] *= row_scale[r] * col_scale[c]
    const float *col_scale;
    int *status;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// bounded wait for the phase with parity `parity`; false on time-out
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < TC_SPIN_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int c0, int c1, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(const void *p) {
    const uint64_t a = smem_u32(p);
    uint64_t d = (a >> 4) & 0x3FFFull;
    d |= (uint64_t)1 << 16;               // leading byte offset (unused with 128B swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;     // stride byte offset
    d |= (uint64_t)1 << 46;               // version
    d |= (uint64_t)2 << 61;               // SWIZZLE_128B
    return d;
}

// instruction descriptor, D float32, A and B K-major, M = 128.
// FP8 = 0: kind::f16 with bf16 operands (format 1); FP8 = 1: kind::f8f6f4 with e4m3 (format 0).
template <int FP8>
__host__ __device__ __forceinline__ uint32_t idesc_tc(int M, int N) {
    const uint32_t fmt = FP8 ? 0u : 1u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// FP8 = 0: bf16 operands, 64 elements (128 B) per K block, K = 16 per MMA;
// FP8 = 1: e4m3 operands, 128 elements (128 B) per K block, K = 32 per MMA.
template <int FP8>
__global__ void __launch_bounds__(128, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, const TcParams p) {
    constexpr int KBLK = FP8 ? 128 : 64;  // elements per 128-byte swizzle row
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int BN = p.BN;
    const uint32_t a_bytes = TC_BM * 128, b_bytes = (uint32_t)BN * 128;
    const uint32_t stage_bytes = a_bytes + b_bytes;  // multiple of 1024 (BN % 16 == 0... and BN*128 % 1024 == 0)
    uint64_t *full = reinterpret_cast<uint64_t *>(base + TC_STAGES * stage_bytes);
    uint64_t *empty = full + TC_STAGES;
    uint64_t *accum = empty + TC_STAGES;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(accum + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * BN;
    const int total_kb = (p.K + KBLK - 1) / KBLK;
    const int kb0 = blockIdx.z * p.kb_per_split;
    const int nkb = min(kb0 + p.kb_per_split, total_kb) - kb0;
    uint32_t tcols = 32;
    while (tcols < (uint32_t)BN) tcols <<= 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(accum, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (nkb > 0 && warp == 0 && lane == 0) {
        // producer
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % TC_STAGES;
            if (kb >= TC_STAGES && !mbar_wait(empty + s, ((kb / TC_STAGES) - 1) & 1)) {
                *abort_flag = 1;
                atomicOr(p.status, ST_TIMEOUT);
                break;
            }
            if (*abort_flag) break;
            uint8_t *sa = base + s * stage_bytes;
            mbar_expect_tx(full + s, stage_bytes);
            const int kx = (kb0 + kb) * KBLK;  // a multiple of 128 bytes
            tma_load_2d(sa, &ta, kx, m0, full + s);
            tma_load_2d(sa + a_bytes, &tb, kx, n0, full + s);
        }
    } else if (nkb > 0 && warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = idesc_tc<FP8>(TC_BM, BN);
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % TC_STAGES;
            if (!mbar_wait(full + s, (kb / TC_STAGES) & 1)) {
                *abort_flag = 1;
                atomicOr(p.status, ST_TIMEOUT);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint8_t *sa = base + s * stage_bytes;
#pragma unroll
            for (int k = 0; k < 4; ++k) {  // 4 MMAs of 32 bytes of K each per 128-byte row
                const uint64_t ad = sdesc(sa + 32 * k);
                const uint64_t bd = sdesc(sa + a_bytes + 32 * k);
                const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
                if (FP8)
                    asm volatile(
                        "{\n\t.reg .pred p;\n\t"
                        "setp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                        : "memory");
                else
                    asm volatile(
                        "{\n\t.reg .pred p;\n\t"
                        "setp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                        : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(empty + s))
                         : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(accum))
                     : "memory");
    }
    __syncwarp();

    // epilogue: TMEM lane = output row of the tile, one warp per 32 lanes
    bool ok = nkb > 0 && mbar_wait(accum, 0) && !*abort_flag;
    if (nkb > 0 && !ok && threadIdx.x == 0) atomicOr(p.status, ST_TIMEOUT);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // each warp moves its 32 rows through a 32 x 33 float slab in the (now idle) stage memory,
        // 32 columns at a time, so that every global store instruction writes one 128-byte row
        // segment
        float *slab = reinterpret_cast<float *>(base) + warp * 32 * 33;
        const int row0 = m0 + warp * 32;
        for (int c0 = 0; c0 < BN; c0 += 32) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int cc = c0 + 16 * h;
                uint32_t r[16];
                if (cc < BN) {
                    const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc;
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                        "%15}, [%16];"
                        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                          "=r"(r[14]), "=r"(r[15])
                        : "r"(addr));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) slab[lane * 33 + 16 * h + j] = cc < BN ? __uint_as_float(r[j]) : 0.f;
            }
            __syncwarp();
            const int col = n0 + c0 + lane;
            const float cs = (p.row_scale && col < p.N) ? p.col_scale[col] : 1.f;
            for (int rr = 0; rr < 32; ++rr) {
                const int row = row0 + rr;
                if (row < p.M && c0 + lane < BN && col < p.N) {
                    float v = slab[rr * 33 + lane];
                    if (p.row_scale) v *= p.row_scale[row] * cs;
                    if (p.partial)
                        p.partial[((int64_t)blockIdx.z * p.M + row) * p.N + col] = v;
                    else
                        p.C[(int64_t)row * p.ldc + col] = v;
                }
            }
            __syncwarp();
        }
    } else if (nkb > 0 && warp == 0 && lane == 0) {
        // drain: wait (bounded) for the copies this CTA may still have in flight
        for (int s = 0; s < TC_STAGES && s < nkb; ++s) mbar_wait(full + s, 0);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
}

// ---------------------------------------------------------------------------------------------
// Projection Y = X P^T with X read as float32 and converted to bf16 inside the kernel (no bf16
// copy of X in HBM), P as a bf16 copy loaded by TMA.  Persistent: CTA c takes the 128-row tiles
// c, c + G, ...; the accumulator is double-buffered in tensor memory so that the epilogue of one
// tile overlaps the main loop of the next.
//   warp 9    : lane 0 streams the float32 X blocks (128 rows x 64 columns, 32 KB, no swizzle)
//               by TMA into a 3-deep staging ring
//   warps 4-7 : converters, 128 threads: per K block, 8 chunks of 8 floats each read from the
//               staging buffer -> 8 bf16 -> one 16-byte store at the 128-byte-swizzle position
//               (row r, chunk c) -> r * 128 + ((c ^ (r & 7)) << 4) of the operand stage, the
//               layout TMA would write; the first converter thread also starts the TMA of the
//               stage's P tile
//   warp 8    : TMEM allocation; lane 0 issues tcgen05.mma (M 128, N BN, K 16) and the commits
//   warps 0-3 : epilogue, warp w owns TMEM lanes (= tile rows) 32w .. 32w + 31
// Barriers: sfull[t] (X block bytes), sempty[t] (128 converter arrivals), full[s] (128 converter
// arrivals + the P tile's bytes), empty[s] (MMA commit), tfull[b] (MMA commit after a tile),
// tempty[b] (128 epilogue arrivals).  Every wait is bounded.
constexpr int PF_THREADS = 320, PF_XSTAGES = 3;
constexpr uint32_t PF_XBYTES = 128 * 64 * 4;

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_tx_only(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

struct PfParams {
    int M, K, N, BN;  // N = d (<= 256), BN = round_up(N, 16)
    int stages;       // operand stages (2 or 3)
    float *Y;         // M x ldy float32; columns N .. ldy-1 written with zeros
    int ldy;
    int *status;
};

__global__ void __launch_bounds__(PF_THREADS, 1)
    proj_f32in_kernel(const __grid_constant__ CUtensorMap tx, const __grid_constant__ CUtensorMap tb,
                      const PfParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int BN = p.BN, PS = p.stages;
    const uint32_t a_bytes = TC_BM * 128, b_bytes = (uint32_t)BN * 128;
    const uint32_t stage_bytes = a_bytes + b_bytes;
    uint8_t *xstage = base + PS * stage_bytes;  // PF_XSTAGES x 32 KB
    uint64_t *full = reinterpret_cast<uint64_t *>(xstage + PF_XSTAGES * PF_XBYTES);
    uint64_t *empty = full + 4;
    uint64_t *sfull = empty + 4;
    uint64_t *sempty = sfull + PF_XSTAGES;
    uint64_t *tfull = sempty + PF_XSTAGES;
    uint64_t *tempty = tfull + 2;
    uint64_t *drain = tempty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles = (p.M + TC_BM - 1) / TC_BM;
    const int nkb = (p.K + 63) / 64;
    const int my_tiles = (int)blockIdx.x < tiles ? (tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int64_t total = (int64_t)my_tiles * nkb;  // this CTA's K blocks, g = 0 .. total - 1

    if (threadIdx.x == 0) {
        for (int s = 0; s < PS; ++s) {
            mbar_init(full + s, 128);
            mbar_init(empty + s, 1);
        }
        for (int t = 0; t < PF_XSTAGES; ++t) {
            mbar_init(sfull + t, 1);
            mbar_init(sempty + t, 128);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull + b, 1);
            mbar_init(tempty + b, 128);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 9) {
        // ---- X producer
        if (lane == 0) {
            for (int64_t g = 0; g < total; ++g) {
                const int t = (int)(g % PF_XSTAGES);
                const int64_t w = g / PF_XSTAGES;
                if (w > 0 && !mbar_wait(sempty + t, (uint32_t)((w - 1) & 1))) {
                    *abort_flag = 1;
                    atomicOr(p.status, ST_TIMEOUT);
                }
                if (*abort_flag) {
                    // drain: the copies already started must land before the CTA exits
                    for (int64_t q = std::max<int64_t>(0, g - PF_XSTAGES); q < g; ++q)
                        mbar_wait(sfull + (int)(q % PF_XSTAGES), (uint32_t)((q / PF_XSTAGES) & 1));
                    break;
                }
                const int tile = (int)blockIdx.x + (int)(g / nkb) * (int)gridDim.x;
                mbar_expect_tx(sfull + t, PF_XBYTES);
                tma_load_2d(xstage + (size_t)t * PF_XBYTES, &tx, (int)(g % nkb) * 64, tile * TC_BM, sfull + t);
            }
        }
        __syncwarp();
    } else if (warp >= 4 && warp < 8) {
        // ---- converters
        const int ct = threadIdx.x - 128;
        for (int64_t g = 0; g < total; ++g) {
            const int t = (int)(g % PF_XSTAGES);
            const int s = (int)(g % PS);
            const int64_t u = g / PS;
            bool ok = !*abort_flag && mbar_wait(sfull + t, (uint32_t)((g / PF_XSTAGES) & 1));
            float4 v[16];
            if (ok) {
                const uint8_t *xs = xstage + (size_t)t * PF_XBYTES;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int ci = ct + 128 * j;
                    const int r = ci >> 3, c = ci & 7;
                    const float4 *src = reinterpret_cast<const float4 *>(xs + r * 256 + 32 * c);
                    v[2 * j] = src[0];
                    v[2 * j + 1] = src[1];
                }
            }
            mbar_arrive(sempty + t);  // the staging block is in registers (or abandoned)
            if (ok && u > 0) ok = mbar_wait(empty + s, (uint32_t)((u - 1) & 1));
            if (!ok || *abort_flag) {
                *abort_flag = 1;
                atomicOr(p.status, ST_TIMEOUT);
                break;
            }
            uint8_t *sa = base + s * stage_bytes;
            if (ct == 0) {
                mbar_tx_only(full + s, b_bytes);
                tma_load_2d(sa + a_bytes, &tb, (int)(g % nkb) * 64, 0, full + s);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int ci = ct + 128 * j;
                const int r = ci >> 3, c = ci & 7;
                uint4 o;
                o.x = pack_bf16x2(v[2 * j].x, v[2 * j].y);
                o.y = pack_bf16x2(v[2 * j].z, v[2 * j].w);
                o.z = pack_bf16x2(v[2 * j + 1].x, v[2 * j + 1].y);
                o.w = pack_bf16x2(v[2 * j + 1].z, v[2 * j + 1].w);
                *reinterpret_cast<uint4 *>(sa + r * 128 + ((c ^ (r & 7)) << 4)) = o;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(full + s);
        }
    } else if (warp == 8) {
        // ---- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_tc<0>(TC_BM, BN);
            int64_t g = 0;
            for (int tc = 0; tc < my_tiles && !*abort_flag; ++tc) {
                const int b = tc & 1, v = tc >> 1;
                if (v > 0 && !mbar_wait(tempty + b, (uint32_t)((v - 1) & 1))) {
                    *abort_flag = 1;
                    atomicOr(p.status, ST_TIMEOUT);
                    break;
                }
                const uint32_t acc_addr = tmem + (uint32_t)(b * 256);
                bool ok = true;
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int s = (int)(g % PS);
                    if (!mbar_wait(full + s, (uint32_t)((g / PS) & 1)) || *abort_flag) {
                        *abort_flag = 1;
                        atomicOr(p.status, ST_TIMEOUT);
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    uint8_t *sa = base + s * stage_bytes;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint64_t ad = sdesc(sa + 32 * k);
                        const uint64_t bd = sdesc(sa + a_bytes + 32 * k);
                        const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\t"
                            "setp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc_addr),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                            : "memory");
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(empty + s))
                                 : "memory");
                }
                if (!ok) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(tfull + b))
                             : "memory");
            }
            // every MMA this thread issued has completed once `drain` flips
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(drain))
                         : "memory");
            if (!mbar_wait(drain, 0)) atomicOr(p.status, ST_TIMEOUT);
        }
        __syncwarp();
    } else {
        // ---- epilogue: tile row = TMEM lane; each warp moves its 32 rows through a 32 x 33
        // float slab in shared memory, 32 columns at a time, so that every global store
        // instruction writes one whole 128-byte row segment
        float *slab = reinterpret_cast<float *>(tmem_slot + 2) + warp * 32 * 33;
        for (int tc = 0; tc < my_tiles; ++tc) {
            const int tile = (int)blockIdx.x + tc * (int)gridDim.x;
            const int b = tc & 1, v = tc >> 1;
            const bool ok = !*abort_flag && mbar_wait(tfull + b, (uint32_t)(v & 1));
            if (!ok) {
                *abort_flag = 1;
                atomicOr(p.status, ST_TIMEOUT);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int row0 = tile * TC_BM + warp * 32;
            for (int c0 = 0; c0 < p.ldy; c0 += 32) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int cc = c0 + 16 * h;
                    uint32_t r[16];
                    if (cc < BN) {
                        const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * 256 + cc);
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                              "=r"(r[14]), "=r"(r[15])
                            : "r"(addr));
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        slab[lane * 33 + 16 * h + j] = (cc + j < p.N) ? __uint_as_float(r[j]) : 0.f;
                }
                __syncwarp();
                const int col = c0 + lane;
                for (int rr = 0; rr < 32; ++rr) {
                    const int row = row0 + rr;
                    if (row < p.M && col < p.ldy) p.Y[(int64_t)row * p.ldy + col] = slab[rr * 33 + lane];
                }
                __syncwarp();
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(tempty + b);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 8)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// ---------------------------------------------------------------------------------------------
// C = A B^T in float32-accurate tf32x3 form on the tensor cores (tcgen05.mma kind::tf32), for the
// differentiation form of the OOD loss.  Each operand comes as a tf32 pair (hi = tf32(v),
// lo = tf32(v - hi), both exact in tf32) and every tile product is hi_a hi_b + hi_a lo_b + lo_a hi_b:
// three tf32 MMAs that keep about 21 bits of the float32 products (the tf32 unit reads only the
// top 19 bits of a float; one tf32 product alone is biased by its truncation).  Float32 tiles go
// from HBM to shared memory by TMA (128-byte swizzle, 32 floats per row) and straight into the MMA.
// Persistent over work items = (K split, 128 x 256 tile), items t = c, c + G, ...; two TMEM
// accumulators (512 columns) let the epilogue of one item overlap the main loop of the next.
// Rows and K columns past the operands' extents are zero-filled by TMA and add nothing.
//   warp 0, lane 0 : TMA producer (2-stage ring of A hi / lo 128 x 32 and B hi / lo 256 x 32 tiles)
//   warp 1         : TMEM allocation; lane 0 issues the MMAs (M 128, N 256, K 8) and commits
//   warps 2-5 (PAIR_SQ) or 2-9 (the others): epilogue; warp w reads TMEM lanes 32 (w % 4) .. (rows
//                    of C), the 256 columns or, with eight warps, half of them each; by MODE:
//     PAIR_SQ : sum of squares of its rows (float32 per 16 columns, then FP64), one FP64 partial
//               per CTA -- the pair loss, with A = Qt (qt_j = q_j - B^T A q_j) and B = X, so that
//               r_ij = qt_j^T x_i carries no cancellation inside the tile products;
//     PAIR_R  : the tile as tf32 hi / lo pairs twice: C^T (lanes write consecutive rows of C, so
//               each column is one coalesced run) and C row-major (through a 32 x 33 shared-memory
//               slab per warp, one coalesced 128-byte run per row) -- the residual matrix R and
//               R^T, operands of the two gradient contractions;
//     PAIR_T  : C^T of split s into out + s * split_stride (float32, pitch ldo), added to what is
//               there when `accumulate` -- R X' and R^T Q' with the d-wide side as M.
constexpr int PL_STAGES = 2, PL_BN = 256;
constexpr int PAIR_SQ = 0, PAIR_R = 1, PAIR_T = 2;

struct PairOut {
    double *partial = nullptr;                                      // PAIR_SQ
    float *ch = nullptr, *cl = nullptr, *th = nullptr, *tl = nullptr;  // PAIR_R
    int64_t ldc = 0, ldt = 0;
    float *out = nullptr;                                           // PAIR_T
    int64_t ldo = 0, split_stride = 0;
    int accumulate = 0;
};

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    return __uint_as_float(h);
}

// 16 consecutive TMEM columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld16(uint32_t addr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(addr));
}

// Tile t -> (m0, n0): groups of PAIR_GROUP row tiles, column-major inside a group, so that the CTAs
// running at one time share a few A row tiles and each B column tile is read by up to PAIR_GROUP of
// them close together (B re-read mt / PAIR_GROUP times from DRAM instead of up to mt times once the
// L2 is busy with the stores of the R epilogue); the last group may hold fewer rows.
constexpr int PAIR_GROUP = 16;
__device__ __forceinline__ void pair_tile(int64_t tile, int mt, int nt, int &m0, int &n0) {
    const int64_t per = (int64_t)PAIR_GROUP * nt;
    const int64_t g = tile / per, r = tile % per;
    const int gm = (int)min((int64_t)PAIR_GROUP, (int64_t)mt - g * PAIR_GROUP);
    m0 = (int)((g * PAIR_GROUP + r % gm) * TC_BM);
    n0 = (int)((r / gm) * PL_BN);
}

// epilogue warps: four for the light sum of squares, eight (two per TMEM lane quarter, half the
// columns each) where the epilogue stores the tile
template <int MODE>
constexpr int pair_epi_warps() { return MODE == PAIR_SQ ? 4 : 8; }

template <int MODE>
__global__ void __launch_bounds__(64 + 32 * pair_epi_warps<MODE>(), 1)
    pair_tf32_kernel(const __grid_constant__ CUtensorMap tah, const __grid_constant__ CUtensorMap tal,
                     const __grid_constant__ CUtensorMap tbh, const __grid_constant__ CUtensorMap tbl, int M, int N,
                     int K, int splits, int kps, const PairOut o, int *__restrict__ status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    // stage: A hi | A lo | B hi | B lo
    const uint32_t a_bytes = TC_BM * 128, b_bytes = PL_BN * 128, stage_bytes = 2 * (a_bytes + b_bytes);
    uint64_t *full = reinterpret_cast<uint64_t *>(base + PL_STAGES * stage_bytes);
    uint64_t *empty = full + PL_STAGES;
    uint64_t *tfull = empty + PL_STAGES;
    uint64_t *tempty = tfull + 2;
    uint64_t *drain = tempty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    constexpr int EW = pair_epi_warps<MODE>();
    // after the barriers: PAIR_SQ's FP64 reduction slots, or the others' 32 x 33 slabs (one per warp)
    double *red = reinterpret_cast<double *>(base + PL_STAGES * stage_bytes + 256);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = (M + TC_BM - 1) / TC_BM, nt = (N + PL_BN - 1) / PL_BN;
    const int64_t tiles = (int64_t)mt * nt, items = tiles * splits;
    const int nkb = (K + 31) / 32;
    const int my_items = (int64_t)blockIdx.x < items ? (int)((items - 1 - blockIdx.x) / gridDim.x) + 1 : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < PL_STAGES; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull + b, 1);
            mbar_init(tempty + b, 32 * EW);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    double acc = 0.0;

    if (warp == 0) {
        if (lane == 0) {
            int64_t g = 0;
            for (int it = 0; it < my_items && !*abort_flag; ++it) {
                const int64_t item = blockIdx.x + (int64_t)it * gridDim.x;
                int m0, n0;
                pair_tile(item % tiles, mt, nt, m0, n0);
                const int kb0 = (int)(item / tiles) * kps, kb1 = min(nkb, kb0 + kps);
                for (int kb = kb0; kb < kb1; ++kb, ++g) {
                    const int s = (int)(g % PL_STAGES);
                    const int64_t u = g / PL_STAGES;
                    if (u > 0 && !mbar_wait(empty + s, (uint32_t)((u - 1) & 1))) {
                        *abort_flag = 1;
                        atomicOr(status, ST_TIMEOUT);
                        break;
                    }
                    uint8_t *sa = base + s * stage_bytes;
                    mbar_expect_tx(full + s, stage_bytes);
                    tma_load_2d(sa, &tah, kb * 32, m0, full + s);
                    tma_load_2d(sa + a_bytes, &tal, kb * 32, m0, full + s);
                    tma_load_2d(sa + 2 * a_bytes, &tbh, kb * 32, n0, full + s);
                    tma_load_2d(sa + 2 * a_bytes + b_bytes, &tbl, kb * 32, n0, full + s);
                }
            }
            // the copies in flight land before the CTA ends (bounded waits)
            for (int64_t q = std::max<int64_t>(0, g - PL_STAGES); q < g; ++q)
                mbar_wait(full + (int)(q % PL_STAGES), (uint32_t)((q / PL_STAGES) & 1));
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // kind::tf32: A and B format 2 (TF32), D float32, M = 128, N = 256
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(PL_BN >> 3) << 17) |
                                   ((uint32_t)(TC_BM >> 4) << 24);
            int64_t g = 0;
            for (int it = 0; it < my_items && !*abort_flag; ++it) {
                const int64_t item = blockIdx.x + (int64_t)it * gridDim.x;
                const int kb0 = (int)(item / tiles) * kps, kb1 = min(nkb, kb0 + kps);
                const int b = it & 1, v = it >> 1;
                if (v > 0 && !mbar_wait(tempty + b, (uint32_t)((v - 1) & 1))) {
                    *abort_flag = 1;
                    atomicOr(status, ST_TIMEOUT);
                    break;
                }
                const uint32_t acc_addr = tmem + (uint32_t)(b * 256);
                bool ok = true;
                for (int kb = kb0; kb < kb1; ++kb, ++g) {
                    const int s = (int)(g % PL_STAGES);
                    if (!mbar_wait(full + s, (uint32_t)((g / PL_STAGES) & 1)) || *abort_flag) {
                        *abort_flag = 1;
                        atomicOr(status, ST_TIMEOUT);
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    uint8_t *sa = base + s * stage_bytes;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {  // 8 floats (32 bytes) of K per MMA, 4 per 128-byte row
                        const uint64_t ah = sdesc(sa + 32 * k), al = sdesc(sa + a_bytes + 32 * k);
                        const uint64_t bh = sdesc(sa + 2 * a_bytes + 32 * k);
                        const uint64_t bl = sdesc(sa + 2 * a_bytes + b_bytes + 32 * k);
                        const uint64_t ad[3] = {ah, ah, al}, bd[3] = {bh, bl, bh};
#pragma unroll
                        for (int t = 0; t < 3; ++t) {
                            const uint32_t accf = (kb > kb0 || k > 0 || t > 0) ? 1u : 0u;
                            asm volatile(
                                "{\n\t.reg .pred p;\n\t"
                                "setp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc_addr),
                                "l"(ad[t]), "l"(bd[t]), "r"(idesc), "r"(accf)
                                : "memory");
                        }
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(empty + s))
                                 : "memory");
                }
                if (!ok) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(tfull + b))
                             : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(drain))
                         : "memory");
            if (!mbar_wait(drain, 0)) atomicOr(status, ST_TIMEOUT);
        }
        __syncwarp();
    } else {
        // ---- epilogue: warps 2..5 (and 6..9) cover the TMEM lane quarters 2, 3, 0, 1
        const int quarter = warp & 3;
        constexpr int NCW = PL_BN / (EW / 4);  // columns per epilogue warp
        const int cbeg = ((warp - 2) >> 2) * NCW;
        float *slab = reinterpret_cast<float *>(base + PL_STAGES * stage_bytes + 256) + (warp - 2) * 32 * 33;
        for (int it = 0; it < my_items; ++it) {
            const int b = it & 1, v = it >> 1;
            const bool ok = !*abort_flag && mbar_wait(tfull + b, (uint32_t)(v & 1));
            if (!ok) {
                *abort_flag = 1;
                atomicOr(status, ST_TIMEOUT);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int64_t item = blockIdx.x + (int64_t)it * gridDim.x;
            int m0, n0;
            pair_tile(item % tiles, mt, nt, m0, n0);
            const int row0 = m0 + quarter * 32;  // C rows of this warp: row0 .. row0 + 31
            const int row = row0 + lane;
            const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 256);
            if (MODE == PAIR_SQ) {
                for (int c0 = 0; c0 < PL_BN; c0 += 16) {
                    uint32_t r[16];
                    tmem_ld16(tbase + (uint32_t)c0, r);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    float sq = 0.f;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float x = __uint_as_float(r[j]);
                        sq = fmaf(x, x, sq);
                    }
                    acc += (double)sq;
                }
            } else {
                for (int c0 = cbeg; c0 < cbeg + NCW && n0 + c0 < N; c0 += 32) {  // warp-uniform bound
                    uint32_t r[32];
                    tmem_ld16(tbase + (uint32_t)c0, r);
                    tmem_ld16(tbase + (uint32_t)(c0 + 16), r + 16);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    const int ncols = min(32, N - (n0 + c0));
                    if (MODE == PAIR_T) {
                        float *os = o.out + (int64_t)(item / tiles) * o.split_stride;
                        if (row < M) {
#pragma unroll
                            for (int j = 0; j < 32; ++j) {
                                if (j < ncols) {
                                    float *p = os + (int64_t)(n0 + c0 + j) * o.ldo + row;
                                    const float x = __uint_as_float(r[j]);
                                    *p = o.accumulate ? *p + x : x;
                                }
                            }
                        }
                    } else {
                        float hi[32], lo[32];
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const float x = __uint_as_float(r[j]);
                            hi[j] = tf32_rna(x);
                            lo[j] = tf32_rna(__fsub_rn(x, hi[j]));
                        }
                        // C^T: column n0 + c0 + j is row n0 + c0 + j of C^T, the lanes' rows consecutive
                        if (row < M) {
#pragma unroll
                            for (int j = 0; j < 32; ++j) {
                                if (j < ncols) {
                                    const int64_t at = (int64_t)(n0 + c0 + j) * o.ldt + row;
                                    o.th[at] = hi[j];
                                    o.tl[at] = lo[j];
                                }
                            }
                        }
                        // C row-major: lane j of the slab's row r is column n0 + c0 + j of row row0 + r
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
#pragma unroll
                            for (int j = 0; j < 32; ++j) slab[lane * 33 + j] = h ? lo[j] : hi[j];
                            __syncwarp();
                            float *dst = h ? o.cl : o.ch;
                            if (lane < ncols) {
                                for (int rr = 0; rr < 32 && row0 + rr < M; ++rr)
                                    dst[(int64_t)(row0 + rr) * o.ldc + n0 + c0 + lane] = slab[rr * 33 + lane];
                            }
                            __syncwarp();
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(tempty + b);
        }
    }
    // PAIR_SQ: one FP64 partial per CTA, the epilogue threads' sums in a fixed order
    if (MODE == PAIR_SQ && warp >= 2) red[threadIdx.x - 64] = acc;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (MODE == PAIR_SQ && threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < 128; ++i) t += red[i];
        o.partial[blockIdx.x] = t;
    }
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// ---------------------------------------------------------------------------------------------
// Gradient contraction of the pair loss with the residual tiles recomputed, never stored
// (Eq. "leanvec_gradients" written per pair, Sec. 2.2):
//   O[r][:] = sum_c (sum_k Rows[r][k] Cols[c][k]) C[c][:]      (r over a row tile of 128, c over
// column blocks of 128), i.e. U = R X' (Rows = Qt, Cols = X, C = X') or V = R^T Q' (Rows = X,
// Cols = Qt, C = Q'), R = Qt X^T.  Per (row tile, column block):
//   MMA1: S = Rows Cols^T over K = D in bf16x3 form (bf16 hi / lo splits of the float32 operands,
//         hi hi + hi lo + lo hi: kind::f16 MMAs with float32 accumulation in TMEM; the dropped lo lo
//         term and the split remainders are ~2^-17 relative, unbiased);
//   epilogue warps: S (TMEM) -> tf32 hi / lo pair P_hi (in place) and P_lo (TMEM), so that
//   MMA2: O += P C over K = 128 in tf32x3 form with A read from TMEM (kind::tf32) and B = C^T
//         (d x 128, tf32 hi / lo) by TMA.
// S is double-buffered in TMEM (two 128-column buffers), P_lo and the O accumulator take the other
// 256 columns: MMA1 of the next block runs while the epilogue splits this one.  Work items are
// (row tile, range of column blocks); an item's O is written to its split's partial slot.
//   warp 0 lane 0: TMA producer, 3-stage ring of 64 KB stages (MMA1: Rows hi / lo 128 x 64 bf16,
//                  Cols hi / lo 128 x 64 bf16; MMA2: C^T hi / lo, two 32-column blocks each)
//   warp 1: TMEM (512 columns); lane 0 issues MMA1 of block t + 1 before MMA2 of block t
//   warps 2-9: epilogue (warp w: TMEM lanes 32 (w % 4) ..; columns 64 ((w - 2) / 4) .. + 63)
// Every wait is bounded: a time-out sets the status word's TIMEOUT bit and the kernel drains.
constexpr int PFL_STAGES = 3;
constexpr uint32_t PFL_STAGE_BYTES = 65536;
constexpr int PFL_EPI_WARPS = 8;
constexpr int PFL_BC = 128;  // columns per block (the K of MMA2)

struct PflParams {
    int M, N, K, d, dn;  // rows, columns, inner dimension, d, d rounded up to 16 (MMA2's N)
    int cblocks, cbps, splits;
    float *out;          // partial[split][M][d]
    int *status;
};

// 32 consecutive TMEM columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld32(uint32_t addr, uint32_t *r) {
    tmem_ld16(addr, r);
    tmem_ld16(addr + 16, r + 16);
}

// 16 consecutive TMEM columns of this warp's 32 lanes <- r
__device__ __forceinline__ void tmem_st16(uint32_t addr, const uint32_t *r) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            addr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__global__ void __launch_bounds__(64 + 32 * PFL_EPI_WARPS, 1)
    pair_flash_kernel(const __grid_constant__ CUtensorMap trh, const __grid_constant__ CUtensorMap trl,
                      const __grid_constant__ CUtensorMap tch, const __grid_constant__ CUtensorMap tcl,
                      const __grid_constant__ CUtensorMap tth, const __grid_constant__ CUtensorMap ttl,
                      const PflParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(base + PFL_STAGES * PFL_STAGE_BYTES);
    uint64_t *empty = full + PFL_STAGES;
    uint64_t *sfull = empty + PFL_STAGES;  // [2] MMA1 of block t done (buffer t & 1)
    uint64_t *pready = sfull + 2;          // [2] P_hi / P_lo of block t written (256 arrivals)
    uint64_t *m2done = pready + 2;         // MMA2 of a block done (one completion per block)
    uint64_t *odone = m2done + 1;          // the last MMA2 of an item done (one per item)
    uint64_t *ofree = odone + 1;           // O read out (256 arrivals, one completion per item)
    uint64_t *drain = ofree + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = (p.M + TC_BM - 1) / TC_BM;
    const int64_t items = (int64_t)mt * p.splits;
    const int nkb = (p.K + 63) / 64;  // MMA1 stages per block
    const int my_items = (int64_t)blockIdx.x < items ? (int)((items - 1 - blockIdx.x) / gridDim.x) + 1 : 0;
    constexpr uint32_t HALF = 16384;  // 128 rows x 128 bytes: one operand tile of a stage
    const uint32_t ct_box = (uint32_t)p.dn * 128;  // one C^T box (dn rows x 32 floats)

    if (threadIdx.x == 0) {
        for (int s = 0; s < PFL_STAGES; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(sfull + b, 1);
            mbar_init(pready + b, 32 * PFL_EPI_WARPS);
        }
        mbar_init(m2done, 1);
        mbar_init(odone, 1);
        mbar_init(ofree, 32 * PFL_EPI_WARPS);
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    // TMEM columns: S / P_hi buffers 0 and 128, P_lo 256, O 384
    auto item_range = [&](int it, int &r0, int &c0, int &c1, int &split) {
        const int64_t item = blockIdx.x + (int64_t)it * gridDim.x;
        const int rt = (int)(item % mt);
        split = (int)(item / mt);
        r0 = rt * TC_BM;
        c0 = split * p.cbps;
        c1 = min(p.cblocks, c0 + p.cbps);
    };

    if (warp == 0) {
        if (lane == 0) {
            int64_t g = 0;
            bool ok = true;
            auto acquire = [&](int64_t gg) -> uint8_t * {
                const int s = (int)(gg % PFL_STAGES);
                const int64_t u = gg / PFL_STAGES;
                if (u > 0 && !mbar_wait(empty + s, (uint32_t)((u - 1) & 1))) return nullptr;
                return base + s * PFL_STAGE_BYTES;
            };
            auto load_ct = [&](int cb) -> bool {  // MMA2's operands of block cb: two stages
                for (int h = 0; h < 2; ++h, ++g) {
                    uint8_t *sa = acquire(g);
                    if (!sa || *abort_flag) return false;
                    uint64_t *f = full + (int)(g % PFL_STAGES);
                    mbar_expect_tx(f, 4 * ct_box);
                    const int x = cb * PFL_BC + h * 64;
                    tma_load_2d(sa, &tth, x, 0, f);
                    tma_load_2d(sa + ct_box, &tth, x + 32, 0, f);
                    tma_load_2d(sa + 2 * ct_box, &ttl, x, 0, f);
                    tma_load_2d(sa + 3 * ct_box, &ttl, x + 32, 0, f);
                }
                return true;
            };
            int prev = -1;
            for (int it = 0; it < my_items && ok; ++it) {
                int r0, c0, c1, split;
                item_range(it, r0, c0, c1, split);
                for (int cb = c0; cb < c1 && ok; ++cb) {
                    for (int kb = 0; kb < nkb; ++kb, ++g) {
                        uint8_t *sa = acquire(g);
                        if (!sa || *abort_flag) {
                            ok = false;
                            break;
                        }
                        uint64_t *f = full + (int)(g % PFL_STAGES);
                        mbar_expect_tx(f, PFL_STAGE_BYTES);
                        tma_load_2d(sa, &trh, kb * 64, r0, f);
                        tma_load_2d(sa + HALF, &trl, kb * 64, r0, f);
                        tma_load_2d(sa + 2 * HALF, &tch, kb * 64, cb * PFL_BC, f);
                        tma_load_2d(sa + 3 * HALF, &tcl, kb * 64, cb * PFL_BC, f);
                    }
                    if (ok && prev >= 0) ok = load_ct(prev);
                    prev = cb;
                }
            }
            if (ok && prev >= 0) ok = load_ct(prev);
            if (!ok) {
                *abort_flag = 1;
                atomicOr(p.status, ST_TIMEOUT);
            }
            // the copies in flight land before the CTA ends (bounded waits)
            for (int64_t q = std::max<int64_t>(0, g - PFL_STAGES); q < g; ++q)
                mbar_wait(full + (int)(q % PFL_STAGES), (uint32_t)((q / PFL_STAGES) & 1));
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA1: kind::f16 (bf16 A / B), M = 128, N = 128; MMA2: kind::tf32, M = 128, N = dn
            const uint32_t id1 = idesc_tc<0>(TC_BM, PFL_BC);
            const uint32_t id2 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(p.dn >> 3) << 17) |
                                 ((uint32_t)(TC_BM >> 4) << 24);
            int64_t g = 0;
            int64_t T = 0;  // blocks issued (MMA1)
            bool ok = true;
            auto take = [&]() -> uint8_t * {
                const int s = (int)(g % PFL_STAGES);
                if (!mbar_wait(full + s, (uint32_t)((g / PFL_STAGES) & 1)) || *abort_flag) return nullptr;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                return base + s * PFL_STAGE_BYTES;
            };
            // MMA2 of block U (P in buffer U & 1): first = the item's first block (O starts at 0),
            // last = its last (O complete), item_no = the item's index on this CTA
            auto mma2 = [&](int64_t U, bool first, bool last, int item_no) -> bool {
                if (!mbar_wait(pready + (int)(U & 1), (uint32_t)((U >> 1) & 1))) return false;
                if (first && item_no > 0 && !mbar_wait(ofree, (uint32_t)((item_no - 1) & 1))) return false;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t phi = tmem + (uint32_t)((U & 1) * 128), plo = tmem + 256u, o = tmem + 384u;
                for (int h = 0; h < 2; ++h, ++g) {
                    uint8_t *sa = take();
                    if (!sa) return false;
#pragma unroll
                    for (int blk = 0; blk < 2; ++blk) {
#pragma unroll
                        for (int k = 0; k < 4; ++k) {  // 8 tf32 of K per MMA
                            const uint32_t kk = (uint32_t)(h * 64 + blk * 32 + k * 8);
                            const uint64_t bh = sdesc(sa + blk * ct_box + 32 * k);
                            const uint64_t bl = sdesc(sa + (2 + blk) * ct_box + 32 * k);
                            const uint32_t ad[3] = {phi + kk, phi + kk, plo + kk};
                            const uint64_t bd[3] = {bh, bl, bh};
#pragma unroll
                            for (int q = 0; q < 3; ++q) {
                                const uint32_t acc = (first && h == 0 && blk == 0 && k == 0 && q == 0) ? 0u : 1u;
                                asm volatile(
                                    "{\n\t.reg .pred p;\n\t"
                                    "setp.ne.b32 p, %4, 0;\n\t"
                                    "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(o),
                                    "r"(ad[q]), "l"(bd[q]), "r"(id2), "r"(acc)
                                    : "memory");
                            }
                        }
                    }
                    mma_commit(empty + (int)((g) % PFL_STAGES));
                }
                mma_commit(m2done);
                if (last) mma_commit(odone);
                return true;
            };
            int64_t pU = -1;
            bool pfirst = false, plast = false;
            int pitem = 0;
            for (int it = 0; it < my_items && ok; ++it) {
                int r0, c0, c1, split;
                item_range(it, r0, c0, c1, split);
                for (int cb = c0; cb < c1 && ok; ++cb) {
                    // S buffer T & 1 is free once MMA2 of block T - 2 is done
                    if (T >= 2 && !mbar_wait(m2done, (uint32_t)((T - 2) & 1))) {
                        ok = false;
                        break;
                    }
                    const uint32_t sacc = tmem + (uint32_t)((T & 1) * 128);
                    for (int kb = 0; kb < nkb && ok; ++kb, ++g) {
                        uint8_t *sa = take();
                        if (!sa) {
                            ok = false;
                            break;
                        }
#pragma unroll
                        for (int k = 0; k < 4; ++k) {  // 16 bf16 (32 bytes) of K per MMA
                            const uint64_t ah = sdesc(sa + 32 * k), al = sdesc(sa + HALF + 32 * k);
                            const uint64_t bh = sdesc(sa + 2 * HALF + 32 * k), bl = sdesc(sa + 3 * HALF + 32 * k);
                            const uint64_t ad[3] = {ah, ah, al}, bd[3] = {bh, bl, bh};
#pragma unroll
                            for (int q = 0; q < 3; ++q) {
                                const uint32_t acc = (kb > 0 || k > 0 || q > 0) ? 1u : 0u;
                                asm volatile(
                                    "{\n\t.reg .pred p;\n\t"
                                    "setp.ne.b32 p, %4, 0;\n\t"
                                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(sacc),
                                    "l"(ad[q]), "l"(bd[q]), "r"(id1), "r"(acc)
                                    : "memory");
                            }
                        }
                        mma_commit(empty + (int)(g % PFL_STAGES));
                    }
                    if (!ok) break;
                    mma_commit(sfull + (int)(T & 1));
                    if (pU >= 0 && !mma2(pU, pfirst, plast, pitem)) {
                        ok = false;
                        break;
                    }
                    pU = T;
                    pfirst = cb == c0;
                    plast = cb == c1 - 1;
                    pitem = it;
                    ++T;
                }
            }
            if (ok && pU >= 0) ok = mma2(pU, pfirst, plast, pitem);
            if (!ok) {
                *abort_flag = 1;
                atomicOr(p.status, ST_TIMEOUT);
            }
            mma_commit(drain);
            if (!mbar_wait(drain, 0)) atomicOr(p.status, ST_TIMEOUT);
        }
        __syncwarp();
    } else {
        // ---- epilogue: warps 2..9, TMEM lane quarter warp % 4, columns 64 ((warp - 2) / 4) .. + 63
        const int quarter = warp & 3;
        const int cb0 = ((warp - 2) >> 2) * 64;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        int64_t T = 0;
        bool ok = true;
        for (int it = 0; it < my_items && ok; ++it) {
            int r0, c0, c1, split;
            item_range(it, r0, c0, c1, split);
            for (int cb = c0; cb < c1; ++cb, ++T) {
                // S of block T, and P_lo free (MMA2 of block T - 1 done)
                if (*abort_flag || !mbar_wait(sfull + (int)(T & 1), (uint32_t)((T >> 1) & 1)) ||
                    (T >= 1 && !mbar_wait(m2done, (uint32_t)((T - 1) & 1)))) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sb = tmem + lane_off + (uint32_t)((T & 1) * 128);
                const uint32_t lb = tmem + lane_off + 256u;
#pragma unroll 1
                for (int c = cb0; c < cb0 + 64; c += 32) {
                    uint32_t r[32], hi[32], lo[32];
                    tmem_ld32(sb + (uint32_t)c, r);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float x = __uint_as_float(r[j]);
                        const float h = tf32_rna(x);
                        hi[j] = __float_as_uint(h);
                        lo[j] = __float_as_uint(tf32_rna(__fsub_rn(x, h)));
                    }
                    tmem_st16(sb + (uint32_t)c, hi);
                    tmem_st16(sb + (uint32_t)c + 16, hi + 16);
                    tmem_st16(lb + (uint32_t)c, lo);
                    tmem_st16(lb + (uint32_t)c + 16, lo + 16);
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(pready + (int)(T & 1));
            }
            if (!ok) break;
            // the item's O: rows r0 + 32 quarter + lane, columns [cb0 / 2 ..) of d, to its split's slot
            if (*abort_flag || !mbar_wait(odone, (uint32_t)(it & 1))) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int row = r0 + quarter * 32 + lane;
            const int half = (warp - 2) >> 2;
            const int cw = p.dn / 2;  // columns of O per warp (dn is a multiple of 16)
            float *orow = p.out + ((int64_t)split * p.M + row) * p.d;
            for (int c = half * cw; c < half * cw + cw; c += 8) {
                uint32_t r[8];
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                               "=r"(r[7])
                             : "r"(tmem + lane_off + 384u + (uint32_t)c));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (row < p.M) {
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (c + j < p.d) orow[c + j] = __uint_as_float(r[j]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(ofree);
        }
        if (!ok) {
            *abort_flag = 1;
            atomicOr(p.status, ST_TIMEOUT);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// ---------------------------------------------------------------------------------------------
// Float32-accurate projection Y = X P^T on the tensor cores: every operand is split into tf32
// hi = tf32(v) and lo = tf32(v - hi) (both exact in tf32) and a tile product is
// hi_x hi_p + hi_x lo_p + lo_x hi_p, three tcgen05.mma kind::tf32 (about 21 bits of each float32
// product; float32 accumulation in TMEM).  X stays float32 in HBM: warp 9 streams 128 x 32 blocks
// by TMA into a 4-deep staging ring, warps 4-7 split them into the hi / lo operand tiles (128-byte
// swizzle, 32 floats per row: chunk c of row r at r * 128 + ((c ^ (r & 7)) << 4)); P's hi / lo
// tiles (split once by tf32_split_kernel) come by TMA.  Persistent over 128-row tiles with two TMEM
// accumulators; the epilogue (warps 0-3) is proj_f32in_kernel's: shared-memory slabs, coalesced
// row stores, zeros in columns N .. ldy-1.
constexpr int TX_XSTAGES = 4;
constexpr uint32_t TX_XBYTES = 128 * 32 * 4;

__global__ void __launch_bounds__(PF_THREADS, 1)
    proj_tf32x3_kernel(const __grid_constant__ CUtensorMap tx, const __grid_constant__ CUtensorMap tbh,
                       const __grid_constant__ CUtensorMap tbl, const PfParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int BN = p.BN, PS = p.stages;
    // operand stage: A hi | A lo | B hi | B lo (one 32-wide K block)
    const uint32_t a_bytes = TC_BM * 128, b_bytes = (uint32_t)BN * 128;
    const uint32_t stage_bytes = 2 * (a_bytes + b_bytes);
    uint8_t *xstage = base + PS * stage_bytes;  // TX_XSTAGES x 16 KB
    uint64_t *full = reinterpret_cast<uint64_t *>(xstage + TX_XSTAGES * TX_XBYTES);
    uint64_t *empty = full + 2;
    uint64_t *sfull = empty + 2;
    uint64_t *sempty = sfull + TX_XSTAGES;
    uint64_t *tfull = sempty + TX_XSTAGES;
    uint64_t *tempty = tfull + 2;
    uint64_t *drain = tempty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles = (p.M + TC_BM - 1) / TC_BM;
    const int nkb = (p.K + 31) / 32;
    const int my_tiles = (int)blockIdx.x < tiles ? (tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int64_t total = (int64_t)my_tiles * nkb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < PS; ++s) {
            mbar_init(full + s, 128);
            mbar_init(empty + s, 1);
        }
        for (int t = 0; t < TX_XSTAGES; ++t) {
            mbar_init(sfull + t, 1);
            mbar_init(sempty + t, 128);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull + b, 1);
            mbar_init(tempty + b, 128);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 9) {
        // ---- X producer
        if (lane == 0) {
            for (int64_t g = 0; g < total; ++g) {
                const int t = (int)(g % TX_XSTAGES);
                const int64_t w = g / TX_XSTAGES;
                if (w > 0 && !mbar_wait(sempty + t, (uint32_t)((w - 1) & 1))) {
                    *abort_flag = 1;
                    atomicOr(p.status, ST_TIMEOUT);
                }
                if (*abort_flag) {
                    for (int64_t q = std::max<int64_t>(0, g - TX_XSTAGES); q < g; ++q)
                        mbar_wait(sfull + (int)(q % TX_XSTAGES), (uint32_t)((q / TX_XSTAGES) & 1));
                    break;
                }
                const int tile = (int)blockIdx.x + (int)(g / nkb) * (int)gridDim.x;
                mbar_expect_tx(sfull + t, TX_XBYTES);
                tma_load_2d(xstage + (size_t)t * TX_XBYTES, &tx, (int)(g % nkb) * 32, tile * TC_BM, sfull + t);
            }
        }
        __syncwarp();
    } else if (warp >= 4 && warp < 8) {
        // ---- converters: 128 rows x 8 chunks of 4 floats per K block, 8 chunks per thread
        const int ct = threadIdx.x - 128;
        for (int64_t g = 0; g < total; ++g) {
            const int t = (int)(g % TX_XSTAGES);
            const int s = (int)(g % PS);
            const int64_t u = g / PS;
            bool ok = !*abort_flag && mbar_wait(sfull + t, (uint32_t)((g / TX_XSTAGES) & 1));
            float4 v[8];
            if (ok) {
                const uint8_t *xs = xstage + (size_t)t * TX_XBYTES;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int ci = ct + 128 * j;
                    v[j] = *reinterpret_cast<const float4 *>(xs + (ci >> 3) * 128 + 16 * (ci & 7));
                }
            }
            mbar_arrive(sempty + t);
            if (ok && u > 0) ok = mbar_wait(empty + s, (uint32_t)((u - 1) & 1));
            if (!ok || *abort_flag) {
                *abort_flag = 1;
                atomicOr(p.status, ST_TIMEOUT);
                break;
            }
            uint8_t *sa = base + s * stage_bytes;
            if (ct == 0) {
                mbar_tx_only(full + s, 2 * b_bytes);
                tma_load_2d(sa + 2 * a_bytes, &tbh, (int)(g % nkb) * 32, 0, full + s);
                tma_load_2d(sa + 2 * a_bytes + b_bytes, &tbl, (int)(g % nkb) * 32, 0, full + s);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int ci = ct + 128 * j;
                const int r = ci >> 3, c = ci & 7;
                const float x[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
                float hi[4], lo[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    hi[e] = tf32_rna(x[e]);
                    lo[e] = tf32_rna(__fsub_rn(x[e], hi[e]));
                }
                const uint32_t off = r * 128 + ((c ^ (r & 7)) << 4);
                *reinterpret_cast<float4 *>(sa + off) = make_float4(hi[0], hi[1], hi[2], hi[3]);
                *reinterpret_cast<float4 *>(sa + a_bytes + off) = make_float4(lo[0], lo[1], lo[2], lo[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(full + s);
        }
    } else if (warp == 8) {
        // ---- MMA issuer: per K block 4 steps of 8 floats, 3 products each
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                   ((uint32_t)(TC_BM >> 4) << 24);
            int64_t g = 0;
            for (int tc = 0; tc < my_tiles && !*abort_flag; ++tc) {
                const int b = tc & 1, v = tc >> 1;
                if (v > 0 && !mbar_wait(tempty + b, (uint32_t)((v - 1) & 1))) {
                    *abort_flag = 1;
                    atomicOr(p.status, ST_TIMEOUT);
                    break;
                }
                const uint32_t acc_addr = tmem + (uint32_t)(b * 256);
                bool ok = true;
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int s = (int)(g % PS);
                    if (!mbar_wait(full + s, (uint32_t)((g / PS) & 1)) || *abort_flag) {
                        *abort_flag = 1;
                        atomicOr(p.status, ST_TIMEOUT);
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    uint8_t *sa = base + s * stage_bytes;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint64_t ah = sdesc(sa + 32 * k), al = sdesc(sa + a_bytes + 32 * k);
                        const uint64_t bh = sdesc(sa + 2 * a_bytes + 32 * k);
                        const uint64_t bl = sdesc(sa + 2 * a_bytes + b_bytes + 32 * k);
                        const uint64_t ad[3] = {ah, ah, al}, bd[3] = {bh, bl, bh};
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            const uint32_t accf = (kb > 0 || k > 0 || q > 0) ? 1u : 0u;
                            asm volatile(
                                "{\n\t.reg .pred p;\n\t"
                                "setp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc_addr),
                                "l"(ad[q]), "l"(bd[q]), "r"(idesc), "r"(accf)
                                : "memory");
                        }
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(empty + s))
                                 : "memory");
                }
                if (!ok) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(tfull + b))
                             : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(drain))
                         : "memory");
            if (!mbar_wait(drain, 0)) atomicOr(p.status, ST_TIMEOUT);
        }
        __syncwarp();
    } else {
        // ---- epilogue: tile row = TMEM lane; each warp moves its 32 rows through a 32 x 33
        // float slab in shared memory, 32 columns at a time, so that every global store
        // instruction writes one whole 128-byte row segment
        float *slab = reinterpret_cast<float *>(tmem_slot + 2) + warp * 32 * 33;
        for (int tc = 0; tc < my_tiles; ++tc) {
            const int tile = (int)blockIdx.x + tc * (int)gridDim.x;
            const int b = tc & 1, v = tc >> 1;
            const bool ok = !*abort_flag && mbar_wait(tfull + b, (uint32_t)(v & 1));
            if (!ok) {
                *abort_flag = 1;
                atomicOr(p.status, ST_TIMEOUT);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int row0 = tile * TC_BM + warp * 32;
            for (int c0 = 0; c0 < p.ldy; c0 += 32) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int cc = c0 + 16 * h;
                    uint32_t r[16];
                    if (cc < BN) {
                        const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * 256 + cc);
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                              "=r"(r[14]), "=r"(r[15])
                            : "r"(addr));
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        slab[lane * 33 + 16 * h + j] = (cc + j < p.N) ? __uint_as_float(r[j]) : 0.f;
                }
                __syncwarp();
                const int col = c0 + lane;
                for (int rr = 0; rr < 32; ++rr) {
                    const int row = row0 + rr;
                    if (row < p.M && col < p.ldy) p.Y[(int64_t)row * p.ldy + col] = slab[rr * 33 + lane];
                }
                __syncwarp();
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(tempty + b);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 8)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// sum of the split-K partials in a fixed order
__global__ void splitk_reduce_kernel(const float *__restrict__ part, int splits, int M, int N, float *__restrict__ C,
                                     int ldc) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)M * N) return;
    const int r = (int)(t / N), c = (int)(t % N);
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += part[(int64_t)z * M * N + t];
    C[(int64_t)r * ldc + c] = s;
}

// float32 rows (n x D, stride D) -> bf16 rows (n x ldo, zero-padded)
__global__ void cast_bf16_kernel(const float *__restrict__ X, int64_t n, int D, __nv_bfloat16 *__restrict__ Y, int ldo) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * ldo) return;
    const int64_t r = t / ldo;
    const int c = (int)(t % ldo);
    Y[t] = __float2bfloat16_rn(c < D ? X[r * D + c] : 0.f);
}

// The same with 16-byte accesses (D % 8 == 0, ldo == D, 16-byte aligned X and Y): each thread
// converts 8 consecutive floats (two float4 loads) into one 16-byte store.
__global__ void cast_bf16_vec_kernel(const float *__restrict__ X, int64_t total8, __nv_bfloat16 *__restrict__ Y) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total8; t += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(X) + 2 * t);
        const float4 b = __ldg(reinterpret_cast<const float4 *>(X) + 2 * t + 1);
        const __nv_bfloat162 h0 = __floats2bfloat162_rn(a.x, a.y), h1 = __floats2bfloat162_rn(a.z, a.w);
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(b.x, b.y), h3 = __floats2bfloat162_rn(b.z, b.w);
        uint4 o;
        o.x = *reinterpret_cast<const uint32_t *>(&h0);
        o.y = *reinterpret_cast<const uint32_t *>(&h1);
        o.z = *reinterpret_cast<const uint32_t *>(&h2);
        o.w = *reinterpret_cast<const uint32_t *>(&h3);
        reinterpret_cast<uint4 *>(Y)[t] = o;
    }
}

// float32 rows -> e4m3 rows (n x ldo bytes, zero-padded) with per-row scale max|row| / 448;
// one warp per row
__global__ void cast_e4m3_kernel(const float *__restrict__ X, int64_t n, int D, uint8_t *__restrict__ Y, int ldo,
                                 float *__restrict__ scale) {
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= n) return;
    const float *x = X + r * D;
    float amax = 0.f;
    for (int j = lane; j < D; j += 32) amax = fmaxf(amax, fabsf(x[j]));
    for (int o = 16; o; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    const float s = amax > 0.f ? amax / 448.0f : 1.0f;
    const float inv = 1.0f / s;
    for (int j = lane; j < ldo; j += 32)
        Y[r * ldo + j] = j < D ? (uint8_t)__nv_cvt_float_to_fp8(x[j] * inv, __NV_SATFINITE, __NV_E4M3) : (uint8_t)0;
    if (lane == 0) scale[r] = s;
}

// float32 X (n x D) -> bf16 X^T (D x ldo), ldo >= n, zero-padded; 32 x 32 tiles
__global__ void cast_transpose_bf16_kernel(const float *__restrict__ X, int64_t n, int D,
                                           __nv_bfloat16 *__restrict__ Y, int64_t ldo) {
    __shared__ float tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t r = r0 + i;
        const int c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < n && c < D) ? X[r * D + c] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int c = c0 + i;
        const int64_t r = r0 + threadIdx.x;
        if (c < D && r < ldo) Y[(int64_t)c * ldo + r] = __float2bfloat16_rn(tile[threadIdx.x][i]);
    }
}

// float32 X (n x D) -> bf16 X^T (D x ldo) with 64 x 64 tiles, 16-byte loads and stores
// (D % 4 == 0, ldo % 8 == 0, 16-byte aligned X and Y); rows n..ldo-1 of the output are zero.
__global__ void __launch_bounds__(256) cast_transpose_bf16_vec_kernel(const float *__restrict__ X, int64_t n, int D,
                                                                      __nv_bfloat16 *__restrict__ Y, int64_t ldo) {
    __shared__ __align__(16) __nv_bfloat16 tile[64][72];  // [column of X][row of X], 16-byte padded rows
    const int64_t r0 = (int64_t)blockIdx.x * 64;
    const int c0 = blockIdx.y * 64;
    const int t = threadIdx.x;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = t / 16 + 16 * i, c4 = t % 16;
        const int64_t gr = r0 + r;
        const int gc = c0 + 4 * c4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gr < n && gc < D) v = __ldg(reinterpret_cast<const float4 *>(X + gr * D + gc));
        tile[4 * c4 + 0][r] = __float2bfloat16_rn(v.x);
        tile[4 * c4 + 1][r] = __float2bfloat16_rn(v.y);
        tile[4 * c4 + 2][r] = __float2bfloat16_rn(v.z);
        tile[4 * c4 + 3][r] = __float2bfloat16_rn(v.w);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int c = t / 8 + 32 * j, ch = t % 8;
        const int gc = c0 + c;
        const int64_t gr = r0 + 8 * ch;
        if (gc < D && gr < ldo)
            *reinterpret_cast<uint4 *>(Y + (int64_t)gc * ldo + gr) = *reinterpret_cast<const uint4 *>(&tile[c][8 * ch]);
    }
}

// ------------------------------------------------------------------------ host
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    });
    return fn;
}

// 2-D tensor map over rows x cols (cols contiguous, row stride ld elements) of bf16
// (esize 2) or 8-bit (esize 1) elements; 128-byte-wide boxes.
static int make_map(CUtensorMap *map, const void *ptr, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                    int esize) {
    auto fn = encode_fn();
    if (!fn) return fail(LV_ERR_CUDA, "tcgen05 GEMM: cuTensorMapEncodeTiled unavailable");
    if (((uintptr_t)ptr & 15) || (ld * esize) % 16)
        return fail(LV_ERR_ARG, "tcgen05 GEMM: operands must be 16-byte aligned");
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * esize)};
    cuuint32_t box[2] = {(cuuint32_t)(128 / esize), (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(map, esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                    const_cast<void *>(ptr), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(LV_ERR_CUDA, "tcgen05 GEMM: cuTensorMapEncodeTiled failed");
    return LV_OK;
}

static size_t tc_smem(int BN) { return (size_t)TC_STAGES * (TC_BM + BN) * 128 + 256 + 1024; }

// C = A B^T with A (M x K, lda), B (N x K, ldb) device arrays (bf16, or e4m3 when fp8 with
// per-row scales rs (M) and cs (N)); C float32 (ldc).  `work` (nullable) holds split-K
// partials: splits * M * N floats.
static int gemm_tc(int fp8, const void *A, int64_t M, int64_t lda, const void *B, int N, int64_t ldb, int64_t K,
                   float *C, int ldc, int splits, float *work, const float *rs, const float *cs, int *status,
                   cudaStream_t st) {
    if (M <= 0 || N <= 0 || K <= 0) return fail(LV_ERR_ARG, "tcgen05 GEMM: empty operand");
    if (M >= (int64_t)1 << 31 || K >= (int64_t)1 << 31) return fail(LV_ERR_ARG, "tcgen05 GEMM: sizes too large");
    const int esize = fp8 ? 1 : 2, kblk = 128 / esize;
    int BN = N <= 256 ? (int)round_up(N, 16) : 256;
    const int total_kb = (int)((K + kblk - 1) / kblk);
    splits = std::max(1, std::min(splits, total_kb));
    if (splits > 1 && !work) splits = 1;
    const int kbps = (total_kb + splits - 1) / splits;
    splits = (total_kb + kbps - 1) / kbps;
    CUtensorMap ta, tb;
    int rc = make_map(&ta, A, M, K, lda, TC_BM, esize);
    if (rc) return rc;
    rc = make_map(&tb, B, N, K, ldb, BN, esize);
    if (rc) return rc;
    TcParams p;
    p.M = (int)M;
    p.N = N;
    p.K = (int)K;
    p.BN = BN;
    p.kb_per_split = kbps;
    p.C = C;
    p.ldc = ldc;
    p.partial = splits > 1 ? work : nullptr;
    p.row_scale = rs;
    p.col_scale = cs;
    p.status = status;
    const size_t sm = tc_smem(BN);
    dim3 grid((unsigned)((M + TC_BM - 1) / TC_BM), (unsigned)((N + BN - 1) / BN), (unsigned)splits);
    if (fp8) {
        LV_CUDA(cudaFuncSetAttribute(gemm_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        gemm_tc_kernel<1><<<grid, 128, sm, st>>>(ta, tb, p);
    } else {
        LV_CUDA(cudaFuncSetAttribute(gemm_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        gemm_tc_kernel<0><<<grid, 128, sm, st>>>(ta, tb, p);
    }
    LV_CHECK_LAUNCH("gemm_tc_kernel");
    if (splits > 1) {
        splitk_reduce_kernel<<<(unsigned)((M * N + 255) / 256), 256, 0, st>>>(work, splits, (int)M, N, C, ldc);
        LV_CHECK_LAUNCH("splitk_reduce_kernel");
    }
    return LV_OK;
}

int gemm_bf16_tc(const __nv_bfloat16 *A, int64_t M, int64_t lda, const __nv_bfloat16 *B, int N, int64_t ldb, int64_t K,
                 float *C, int ldc, int splits, float *work, int *status, cudaStream_t st) {
    return gemm_tc(0, A, M, lda, B, N, ldb, K, C, ldc, splits, work, nullptr, nullptr, status, st);
}

int launch_cast_bf16(const float *X, int64_t n, int D, __nv_bfloat16 *Y, int ldo, cudaStream_t st) {
    if (D % 8 == 0 && ldo == D && ((uintptr_t)X & 15) == 0 && ((uintptr_t)Y & 15) == 0) {
        const int64_t total8 = n * D / 8;
        const unsigned grid = (unsigned)std::min<int64_t>((total8 + 255) / 256, 152 * 16);
        if (total8 > 0) cast_bf16_vec_kernel<<<grid, 256, 0, st>>>(X, total8, Y);
        LV_CHECK_LAUNCH("cast_bf16_vec_kernel");
        return LV_OK;
    }
    const int64_t tot = n * ldo;
    cast_bf16_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(X, n, D, Y, ldo);
    LV_CHECK_LAUNCH("cast_bf16_kernel");
    return LV_OK;
}

int launch_cast_transpose_bf16(const float *X, int64_t n, int D, __nv_bfloat16 *Y, int64_t ldo, cudaStream_t st) {
    if (D % 4 == 0 && ldo % 8 == 0 && ((uintptr_t)X & 15) == 0 && ((uintptr_t)Y & 15) == 0) {
        dim3 grd((unsigned)((ldo + 63) / 64), (unsigned)((D + 63) / 64));
        cast_transpose_bf16_vec_kernel<<<grd, 256, 0, st>>>(X, n, D, Y, ldo);
        LV_CHECK_LAUNCH("cast_transpose_bf16_vec_kernel");
        return LV_OK;
    }
    dim3 grd((unsigned)((ldo + 31) / 32), (unsigned)((D + 31) / 32));
    cast_transpose_bf16_kernel<<<grd, dim3(32, 8), 0, st>>>(X, n, D, Y, ldo);
    LV_CHECK_LAUNCH("cast_transpose_bf16_kernel");
    return LV_OK;
}

int ensure_ws(void **p, size_t *have, size_t want);

// the fp32-input projection kernel applies: 16-byte aligned rows of X, d <= 256
static bool proj_fused_ok(const float *X, int D, int d) {
    return D % 4 == 0 && ((uintptr_t)X & 15) == 0 && d >= 1 && d <= 256;
}
bool project_bf16_fused_ok(const float *X, int D, int d) { return proj_fused_ok(X, D, d); }

// v -> (hi, lo) = (tf32(v), tf32(v - hi)), round to nearest; both are float32 values whose low 13
// mantissa bits are zero, so the tf32 MMA reads them exactly
__global__ void tf32_split_kernel(const float *__restrict__ v, int64_t len, float *__restrict__ hi,
                                  float *__restrict__ lo) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < len; t += (int64_t)gridDim.x * blockDim.x) {
        const float x = v[t];
        uint32_t h, l;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
        const float r = __fsub_rn(x, __uint_as_float(h));
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(r));
        hi[t] = __uint_as_float(h);
        lo[t] = __uint_as_float(l);
    }
}

int launch_tf32_split(const float *v, int64_t len, float *hi, float *lo, cudaStream_t st) {
    if (len <= 0) return LV_OK;
    tf32_split_kernel<<<(unsigned)std::min<int64_t>((len + 255) / 256, 152 * 32), 256, 0, st>>>(v, len, hi, lo);
    LV_CHECK_LAUNCH("tf32_split_kernel");
    return LV_OK;
}

// Y^T as tf32 pairs: hi / lo (cols x ldt, row-major) of Y (rows x cols, row-major), 32 x 32 tiles
// through shared memory so that both the reads and the writes are coalesced
__global__ void __launch_bounds__(256) transpose_tf32_split_kernel(const float *__restrict__ Y, int64_t rows,
                                                                   int cols, float *__restrict__ hi,
                                                                   float *__restrict__ lo, int64_t ldt) {
    __shared__ float tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int i = ty; i < 32; i += 8) {
        const int64_t r = r0 + i;
        const int c = c0 + tx;
        tile[i][tx] = (r < rows && c < cols) ? Y[r * cols + c] : 0.f;
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const int c = c0 + i;
        const int64_t r = r0 + tx;
        if (c < cols && r < rows) {
            const float x = tile[tx][i];
            const float h = tf32_rna(x);
            hi[(int64_t)c * ldt + r] = h;
            lo[(int64_t)c * ldt + r] = tf32_rna(__fsub_rn(x, h));
        }
    }
}

int launch_transpose_tf32_split(const float *Y, int64_t rows, int cols, float *hi, float *lo, int64_t ldt,
                                cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return LV_OK;
    if (ldt < rows || cols > 65535 * 32) return fail(LV_ERR_ARG, "transpose_tf32_split: bad sizes");
    transpose_tf32_split_kernel<<<dim3((unsigned)((rows + 31) / 32), (unsigned)((cols + 31) / 32)), 256, 0, st>>>(
        Y, rows, cols, hi, lo, ldt);
    LV_CHECK_LAUNCH("transpose_tf32_split_kernel");
    return LV_OK;
}

static int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return sms;
}

// K blocks per split when K is cut into `splits` ranges, and the number of non-empty ranges
static int split_kps(int64_t K, int splits, int *used) {
    const int64_t nkb = (K + 31) / 32;
    const int64_t kps = (nkb + splits - 1) / splits;
    *used = (int)((nkb + kps - 1) / kps);
    return (int)kps;
}

// C = A B^T (A: M x K, pitch lda; B: N x K, pitch ldb; tf32 hi / lo pairs of float32, row-major,
// 16-byte aligned rows) with the epilogue MODE; `grid` persistent CTAs over splits x tiles items
template <int MODE>
static int pair_tf32_launch(const float *Ah, const float *Al, int64_t M, int64_t lda, const float *Bh,
                            const float *Bl, int64_t N, int64_t ldb, int64_t K, int splits, const PairOut &o,
                            int grid, int *status, cudaStream_t st) {
    if (M <= 0 || N <= 0 || K <= 0 || M >= (1ll << 31) || N >= (1ll << 31) || K >= (1ll << 31) || lda < K ||
        ldb < K || lda % 4 || ldb % 4 || splits < 1)
        return fail(LV_ERR_ARG, "tf32x3 pair GEMM: unsupported sizes");
    for (const float *q : {Ah, Al, Bh, Bl})
        if ((uintptr_t)q & 15) return fail(LV_ERR_ARG, "tf32x3 pair GEMM: operands must be 16-byte aligned");
    auto fn = encode_fn();
    if (!fn) return fail(LV_ERR_CUDA, "tf32x3 pair GEMM: cuTensorMapEncodeTiled unavailable");
    CUtensorMap tah, tal, tbh, tbl;
    auto map = [&](CUtensorMap *mp, const float *ptr, int64_t rows, int64_t ld, int box_rows) -> bool {
        cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
        cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
        cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
        cuuint32_t es[2] = {1, 1};
        return fn(mp, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(ptr), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    if (!map(&tah, Ah, M, lda, TC_BM) || !map(&tal, Al, M, lda, TC_BM) || !map(&tbh, Bh, N, ldb, PL_BN) ||
        !map(&tbl, Bl, N, ldb, PL_BN))
        return fail(LV_ERR_CUDA, "tf32x3 pair GEMM: cuTensorMapEncodeTiled failed");
    int used = 0;
    const int kps = split_kps(K, splits, &used);
    // stages, barriers and flags, eight epilogue slabs (or the FP64 reduction slots), alignment slack
    const size_t sm = (size_t)PL_STAGES * 2 * (TC_BM + PL_BN) * 128 + 256 + 8 * 32 * 33 * 4 + 1024;
    LV_CUDA(cudaFuncSetAttribute(pair_tf32_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    pair_tf32_kernel<MODE><<<grid, 64 + 32 * pair_epi_warps<MODE>(), sm, st>>>(tah, tal, tbh, tbl, (int)M, (int)N, (int)K, used, kps, o,
                                                         status);
    LV_CHECK_LAUNCH("pair_tf32_kernel");
    return LV_OK;
}

static int64_t pair_items(int64_t M, int64_t N, int splits) {
    return ((M + TC_BM - 1) / TC_BM) * ((N + PL_BN - 1) / PL_BN) * splits;
}

// Sum of squares of Qt X^T (Qt m x K, X n x K, given as tf32 hi / lo pairs: float32, row-major,
// 16-byte aligned rows, K % 4 == 0) on the tensor cores; writes one FP64 partial per CTA to
// `partial` (at least *nparts entries: call with partial = NULL to get the count) -- the caller
// sums them in order.
int pair_sq_tf32(const float *Qh, const float *Ql, int64_t m, const float *Xh, const float *Xl, int64_t n, int K,
                 double *partial, int *nparts, int *status, cudaStream_t st) {
    if (m <= 0 || n <= 0 || K <= 0 || K % 4 || m >= (1ll << 31) || n >= (1ll << 31))
        return fail(LV_ERR_ARG, "pair_sq_tf32: unsupported sizes");
    const int sms = sm_count();
    if (sms <= 0) return fail(LV_ERR_CUDA, "pair_sq_tf32: no device");
    const int grid = (int)std::min<int64_t>(pair_items(m, n, 1), sms);
    *nparts = grid;
    if (!partial) return LV_OK;
    PairOut o;
    o.partial = partial;
    return pair_tf32_launch<PAIR_SQ>(Qh, Ql, m, K, Xh, Xl, n, K, K, 1, o, grid, status, st);
}

// C = A B^T (M x N) stored as tf32 pairs twice: C row-major in ch / cl (pitch ldc) and C^T in
// th / tl (N x M, pitch ldt)
int pair_r_tf32(const float *Ah, const float *Al, int64_t M, int64_t lda, const float *Bh, const float *Bl, int64_t N,
                int64_t ldb, int64_t K, float *ch, float *cl, int64_t ldc, float *th, float *tl, int64_t ldt,
                int *status, cudaStream_t st) {
    if (!ch || !cl || !th || !tl || ldc < N || ldt < M) return fail(LV_ERR_ARG, "pair_r_tf32: bad output");
    const int sms = sm_count();
    if (sms <= 0) return fail(LV_ERR_CUDA, "pair_r_tf32: no device");
    PairOut o;
    o.ch = ch;
    o.cl = cl;
    o.th = th;
    o.tl = tl;
    o.ldc = ldc;
    o.ldt = ldt;
    const int grid = (int)std::min<int64_t>(pair_items(M, N, 1), sms);
    return pair_tf32_launch<PAIR_R>(Ah, Al, M, lda, Bh, Bl, N, ldb, K, 1, o, grid, status, st);
}

// K splits for gemm_t_tf32 of an M x N output over K: at least four 32-wide K blocks per split and
// about four to eight work items per SM, the count whose last wave of items is fullest (ties: fewer
// splits); the value is the number of partial slots the call writes
// float32 -> bf16 hi / lo pair: hi = bf16(v) (nearest), lo = bf16(v - hi) (nearest); hi + lo keeps
// 16 significant bits of v
__global__ void bf16_split_kernel(const float *__restrict__ v, int64_t len, __nv_bfloat16 *__restrict__ hi,
                                  __nv_bfloat16 *__restrict__ lo) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < len; t += (int64_t)gridDim.x * blockDim.x) {
        const float x = v[t];
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        hi[t] = h;
        lo[t] = __float2bfloat16_rn(__fsub_rn(x, __bfloat162float(h)));
    }
}

int launch_bf16_split(const float *v, int64_t len, __nv_bfloat16 *hi, __nv_bfloat16 *lo, cudaStream_t st) {
    if (len <= 0) return LV_OK;
    const int64_t blocks = std::min<int64_t>((len + 255) / 256, (int64_t)sm_count() * 16);
    bf16_split_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(v, len, hi, lo);
    LV_CHECK_LAUNCH("bf16_split_kernel");
    return LV_OK;
}

// Column splits of pair_flash for M rows and N columns on `grid` CTAs: the number of column ranges
// that minimises the largest per-CTA load (items taken round-robin), with at most max_splits
// ranges; *cbps = column blocks per range.  Returns the number of non-empty ranges.
int pair_flash_splits(int64_t M, int64_t N, int grid, int max_splits, int *cbps) {
    const int64_t mt = (M + TC_BM - 1) / TC_BM, cb = (N + PFL_BC - 1) / PFL_BC;
    int64_t best_cost = -1;
    int best_s = 1, best_c = (int)cb;
    for (int s = 1; s <= std::min<int64_t>(cb, std::max(1, max_splits)); ++s) {
        const int64_t per = (cb + s - 1) / s, used = (cb + per - 1) / per;
        const int64_t items = mt * used, waves = (items + grid - 1) / grid;
        const int64_t cost = waves * per;
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best_s = (int)used;
            best_c = (int)per;
        }
    }
    *cbps = best_c;
    return best_s;
}

// out[split][M][d] = partial sums over column range `split` of (Rows Cols^T) C: Rows (M x K) and
// Cols (N x K) as bf16 hi / lo pairs (row-major, pitch K, K % 8 == 0, 16-byte aligned), C^T
// (d x N, pitch ldt floats) as tf32 hi / lo pairs; d <= 128.  `splits` / `cbps` from
// pair_flash_splits.  The residual tiles are recomputed in the kernel and never stored.
int pair_flash(const __nv_bfloat16 *Rh, const __nv_bfloat16 *Rl, int64_t M, const __nv_bfloat16 *Ch,
               const __nv_bfloat16 *Cl, int64_t N, int K, const float *Th, const float *Tl, int64_t ldt, int d,
               int splits, int cbps, float *out, int *status, cudaStream_t st) {
    if (M <= 0 || N <= 0 || K <= 0 || K % 8 || d < 1 || d > 128 || M >= (1ll << 31) || N >= (1ll << 31) ||
        ldt < N || ldt % 4 || splits < 1 || cbps < 1)
        return fail(LV_ERR_ARG, "pair_flash: unsupported sizes");
    for (const void *q : {(const void *)Rh, (const void *)Rl, (const void *)Ch, (const void *)Cl, (const void *)Th,
                          (const void *)Tl})
        if ((uintptr_t)q & 15) return fail(LV_ERR_ARG, "pair_flash: operands must be 16-byte aligned");
    auto fn = encode_fn();
    if (!fn) return fail(LV_ERR_CUDA, "pair_flash: cuTensorMapEncodeTiled unavailable");
    CUtensorMap trh, trl, tch, tcl, tth, ttl;
    int rc = make_map(&trh, Rh, M, K, K, TC_BM, 2);
    if (!rc) rc = make_map(&trl, Rl, M, K, K, TC_BM, 2);
    if (!rc) rc = make_map(&tch, Ch, N, K, K, PFL_BC, 2);
    if (!rc) rc = make_map(&tcl, Cl, N, K, K, PFL_BC, 2);
    if (rc) return rc;
    const int dn = (d + 15) / 16 * 16;
    auto tmap = [&](CUtensorMap *mp, const float *ptr) -> bool {
        cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)d};
        cuuint64_t strides[1] = {(cuuint64_t)ldt * 4};
        cuuint32_t box[2] = {32, (cuuint32_t)dn};
        cuuint32_t es[2] = {1, 1};
        return fn(mp, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(ptr), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    if (!tmap(&tth, Th) || !tmap(&ttl, Tl)) return fail(LV_ERR_CUDA, "pair_flash: cuTensorMapEncodeTiled failed");
    PflParams p;
    p.M = (int)M;
    p.N = (int)N;
    p.K = K;
    p.d = d;
    p.dn = dn;
    p.cblocks = (int)((N + PFL_BC - 1) / PFL_BC);
    p.cbps = cbps;
    p.splits = splits;
    p.out = out;
    p.status = status;
    if ((int64_t)(splits - 1) * cbps >= p.cblocks) return fail(LV_ERR_ARG, "pair_flash: an empty column range");
    const int64_t items = ((M + TC_BM - 1) / TC_BM) * splits;
    const int grid = (int)std::min<int64_t>(items, std::max(1, sm_count()));
    const size_t sm = (size_t)PFL_STAGES * PFL_STAGE_BYTES + 256 + 1024;
    LV_CUDA(cudaFuncSetAttribute(pair_flash_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    pair_flash_kernel<<<grid, 64 + 32 * PFL_EPI_WARPS, sm, st>>>(trh, trl, tch, tcl, tth, ttl, p);
    LV_CHECK_LAUNCH("pair_flash_kernel");
    return LV_OK;
}

int gemm_t_tf32_splits(int64_t M, int64_t N, int64_t K) {
    const int64_t sms = std::max(1, sm_count());
    const int64_t tiles = pair_items(M, N, 1), nkb = (K + 31) / 32;
    const int64_t lo = std::max<int64_t>(1, std::min<int64_t>((4 * sms + tiles - 1) / tiles, nkb / 4));
    const int64_t hi = std::max<int64_t>(lo, std::min<int64_t>((8 * sms + tiles - 1) / tiles, nkb / 4));
    int best = 1;
    double best_eff = -1.0;
    for (int64_t s = lo; s <= hi; ++s) {
        int used = 0;
        split_kps(K, (int)s, &used);
        const int64_t items = tiles * used, waves = (items + sms - 1) / sms;
        const double eff = (double)items / (double)(waves * sms);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = used;
        }
    }
    return best;
}

// C = A B^T over K in `splits` ranges (gemm_t_tf32_splits' count); split s writes C^T (N x M,
// pitch ldo) to out + s * split_stride, added to what is there when `accumulate`
int gemm_t_tf32(const float *Ah, const float *Al, int64_t M, int64_t lda, const float *Bh, const float *Bl, int64_t N,
                int64_t ldb, int64_t K, float *out, int64_t ldo, int64_t split_stride, int accumulate, int splits,
                int *status, cudaStream_t st) {
    if (!out || ldo < M) return fail(LV_ERR_ARG, "gemm_t_tf32: bad output");
    const int sms = sm_count();
    if (sms <= 0) return fail(LV_ERR_CUDA, "gemm_t_tf32: no device");
    int used = 0;
    split_kps(K, splits, &used);
    PairOut o;
    o.out = out;
    o.ldo = ldo;
    o.split_stride = split_stride;
    o.accumulate = accumulate;
    const int grid = (int)std::min<int64_t>(pair_items(M, N, used), sms);
    return pair_tf32_launch<PAIR_T>(Ah, Al, M, lda, Bh, Bl, N, ldb, K, splits, o, grid, status, st);
}

// workspace bytes of project_bf16 (prec LV_PREC_BF16) or project_fp8 (LV_PREC_FP8)
size_t project_tc_ws_bytes(int prec, int64_t n, int D, int d, const float *X) {
    if (prec == LV_PREC_TF32X3) return 2 * round_up((int64_t)d * D * 4, 256);
    if (prec == LV_PREC_FP8) {
        const int ldx = (int)round_up(D, 16);
        return round_up((int64_t)n * ldx, 256) + round_up((int64_t)d * ldx, 256) + round_up(4 * n, 256) +
               round_up(4 * (int64_t)d, 256);
    }
    const int ldx = (int)round_up(D, 8);
    if (proj_fused_ok(X, D, d)) return round_up((int64_t)d * ldx * 2, 256);
    return round_up((int64_t)n * ldx * 2, 256) + round_up((int64_t)d * ldx * 2, 256);
}

static int project_bf16_fused(const float *X, int64_t n, int D, const float *P, int d, float *Y, int ldy,
                              void **ws, size_t *ws_bytes, int *status, cudaStream_t st) {
    const int ldx = (int)round_up(D, 8);
    int rc = ensure_ws(ws, ws_bytes, round_up((int64_t)d * ldx * 2, 256));
    if (rc) return rc;
    __nv_bfloat16 *Pb = reinterpret_cast<__nv_bfloat16 *>(*ws);
    rc = launch_cast_bf16(P, d, D, Pb, ldx, st);
    if (rc) return rc;
    const int BN = (int)round_up(d, 16);
    CUtensorMap tb, tx;
    rc = make_map(&tb, Pb, d, D, ldx, BN, 2);
    if (rc) return rc;
    {
        // X as float32 blocks of 128 rows x 64 columns (256-byte rows, no swizzle); rows >= n
        // and columns >= D read as zeros
        auto fn = encode_fn();
        if (!fn) return fail(LV_ERR_CUDA, "tcgen05 GEMM: cuTensorMapEncodeTiled unavailable");
        cuuint64_t dims[2] = {(cuuint64_t)D, (cuuint64_t)n};
        cuuint64_t strides[1] = {(cuuint64_t)D * 4};
        cuuint32_t box[2] = {64, (cuuint32_t)TC_BM};
        cuuint32_t es[2] = {1, 1};
        if (fn(&tx, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(X), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return fail(LV_ERR_CUDA, "tcgen05 GEMM: cuTensorMapEncodeTiled failed for the float32 operand");
    }
    PfParams pp;
    pp.M = (int)n;
    pp.K = D;
    pp.N = d;
    pp.BN = BN;
    pp.Y = Y;
    pp.ldy = ldy;
    pp.status = status;
    // fixed: the X staging ring, barriers and flags (256), the epilogue slabs (4 x 32 x 33 floats),
    // alignment slack (1024)
    const size_t stage = (size_t)(TC_BM + BN) * 128,
                 fixed = (size_t)PF_XSTAGES * PF_XBYTES + 256 + 4 * 32 * 33 * 4 + 1024;
    pp.stages = 3 * stage + fixed <= 227 * 1024 ? 3 : 2;
    const size_t sm = pp.stages * stage + fixed;
    int dev = 0, sms = 0;
    LV_CUDA(cudaGetDevice(&dev));
    LV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t tiles = (n + TC_BM - 1) / TC_BM;
    const unsigned grid = (unsigned)std::min<int64_t>(tiles, sms);
    LV_CUDA(cudaFuncSetAttribute(proj_f32in_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    proj_f32in_kernel<<<grid, PF_THREADS, sm, st>>>(tx, tb, pp);
    LV_CHECK_LAUNCH("proj_f32in_kernel");
    return LV_OK;
}

// Y (n x ldy) = X P^T, float32-accurate, on the tensor cores (three tf32 products of hi / lo
// splits); X is split inside the GEMM (16-byte aligned rows, D % 4 == 0, d <= 256), P's hi / lo
// copies live in the caller's workspace (*ws, grown as needed); columns d..ldy-1 zeroed.
int project_tf32x3(const float *X, int64_t n, int D, const float *P, int d, float *Y, int ldy, void **ws,
                   size_t *ws_bytes, int *status, cudaStream_t st) {
    if (!proj_fused_ok(X, D, d)) return fail(LV_ERR_ARG, "tf32x3 projection: needs D % 4 == 0, aligned rows, d <= 256");
    if (n >= (int64_t)1 << 31) return fail(LV_ERR_ARG, "tf32x3 projection: sizes too large");
    const size_t pb = round_up((int64_t)d * D * 4, 256);
    int rc = ensure_ws(ws, ws_bytes, 2 * pb);
    if (rc) return rc;
    float *Ph = reinterpret_cast<float *>(*ws);
    float *Pl = reinterpret_cast<float *>(reinterpret_cast<uint8_t *>(*ws) + pb);
    rc = launch_tf32_split(P, (int64_t)d * D, Ph, Pl, st);
    if (rc) return rc;
    const int BN = (int)round_up(d, 16);
    auto fn = encode_fn();
    if (!fn) return fail(LV_ERR_CUDA, "tcgen05 GEMM: cuTensorMapEncodeTiled unavailable");
    CUtensorMap tx, tbh, tbl;
    auto map = [&](CUtensorMap *mp, const float *ptr, int64_t rows, int box_rows, CUtensorMapSwizzle sw) -> bool {
        cuuint64_t dims[2] = {(cuuint64_t)D, (cuuint64_t)rows};
        cuuint64_t strides[1] = {(cuuint64_t)D * 4};
        cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
        cuuint32_t es[2] = {1, 1};
        return fn(mp, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(ptr), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    if (!map(&tx, X, n, TC_BM, CU_TENSOR_MAP_SWIZZLE_NONE) || !map(&tbh, Ph, d, BN, CU_TENSOR_MAP_SWIZZLE_128B) ||
        !map(&tbl, Pl, d, BN, CU_TENSOR_MAP_SWIZZLE_128B))
        return fail(LV_ERR_CUDA, "tf32x3 projection: cuTensorMapEncodeTiled failed");
    PfParams pp;
    pp.M = (int)n;
    pp.K = D;
    pp.N = d;
    pp.BN = BN;
    pp.Y = Y;
    pp.ldy = ldy;
    pp.status = status;
    // stage: A hi, A lo, B hi, B lo of one 32-wide K block; fixed: X staging ring, barriers and
    // flags, epilogue slabs, alignment slack
    const size_t stage = (size_t)2 * (TC_BM + BN) * 128,
                 fixed = (size_t)TX_XSTAGES * TX_XBYTES + 256 + 4 * 32 * 33 * 4 + 1024;
    pp.stages = 2 * stage + fixed <= 227 * 1024 ? 2 : 1;
    const size_t sm = pp.stages * stage + fixed;
    int dev = 0, sms = 0;
    LV_CUDA(cudaGetDevice(&dev));
    LV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t tiles = (n + TC_BM - 1) / TC_BM;
    const unsigned grid = (unsigned)std::min<int64_t>(tiles, sms);
    LV_CUDA(cudaFuncSetAttribute(proj_tf32x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    proj_tf32x3_kernel<<<grid, PF_THREADS, sm, st>>>(tx, tbh, tbl, pp);
    LV_CHECK_LAUNCH("proj_tf32x3_kernel");
    return LV_OK;
}

// Y (n x ldy) = X P^T with bf16 operands on the tensor cores; columns d..ldy-1 zeroed.
// X is converted to bf16 inside the GEMM when its rows are 16-byte aligned; otherwise the bf16
// copies of X and P live in the caller's workspace (*ws, grown as needed).
int project_bf16(const float *X, int64_t n, int D, const float *P, int d, float *Y, int ldy, void **ws,
                 size_t *ws_bytes, int *status, cudaStream_t st) {
    if (n >= (int64_t)1 << 31) return fail(LV_ERR_ARG, "tcgen05 GEMM: sizes too large");
    if (proj_fused_ok(X, D, d)) return project_bf16_fused(X, n, D, P, d, Y, ldy, ws, ws_bytes, status, st);
    const int ldx = (int)round_up(D, 8);
    const size_t xb = round_up((int64_t)n * ldx * 2, 256), pb = round_up((int64_t)d * ldx * 2, 256);
    int rc = ensure_ws(ws, ws_bytes, xb + pb);
    if (rc) return rc;
    __nv_bfloat16 *Xb = reinterpret_cast<__nv_bfloat16 *>(*ws);
    __nv_bfloat16 *Pb = reinterpret_cast<__nv_bfloat16 *>(reinterpret_cast<uint8_t *>(*ws) + xb);
    rc = launch_cast_bf16(X, n, D, Xb, ldx, st);
    if (rc) return rc;
    rc = launch_cast_bf16(P, d, D, Pb, ldx, st);
    if (rc) return rc;
    if (ldy > d) LV_CUDA(cudaMemset2DAsync(Y + d, (size_t)ldy * 4, 0, (size_t)(ldy - d) * 4, (size_t)n, st));
    return gemm_bf16_tc(Xb, n, ldx, Pb, d, ldx, D, Y, ldy, 1, nullptr, status, st);
}

// Y (n x ldy) = X P^T with e4m3 operands and per-row scales (X rows and P rows), float32
// accumulation on the tensor cores; columns d..ldy-1 zeroed.
int project_fp8(const float *X, int64_t n, int D, const float *P, int d, float *Y, int ldy, void **ws,
                size_t *ws_bytes, int *status, cudaStream_t st) {
    const int ldx = (int)round_up(D, 16);
    const size_t xb = round_up((int64_t)n * ldx, 256), pb = round_up((int64_t)d * ldx, 256);
    const size_t sxb = round_up(4 * n, 256), spb = round_up(4 * (int64_t)d, 256);
    int rc = ensure_ws(ws, ws_bytes, xb + pb + sxb + spb);
    if (rc) return rc;
    uint8_t *base = reinterpret_cast<uint8_t *>(*ws);
    uint8_t *X8 = base, *P8 = base + xb;
    float *sx = reinterpret_cast<float *>(base + xb + pb), *sp = reinterpret_cast<float *>(base + xb + pb + sxb);
    cast_e4m3_kernel<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(X, n, D, X8, ldx, sx);
    cast_e4m3_kernel<<<(unsigned)((d + 7) / 8), 256, 0, st>>>(P, d, D, P8, ldx, sp);
    LV_CHECK_LAUNCH("cast_e4m3_kernel");
    if (ldy > d) LV_CUDA(cudaMemset2DAsync(Y + d, (size_t)ldy * 4, 0, (size_t)(ldy - d) * 4, (size_t)n, st));
    return gemm_tc(1, X8, n, ldx, P8, d, ldx, D, Y, ldy, 1, nullptr, sx, sp, status, st);
}

// K (D x D) = X^T X over the n rows of X with bf16 operands (X^T staged in bf16).
// ---------------------------------------------------------------------------------------------
// Second moment K = X^T X (Sec. 2.2 "Efficiency") with the float32 rows of X rounded to bf16
// inside the GEMM (bf16 products, float32 accumulation -- the operand rounding of the bf16 path
// through a converted copy of X, without the copy).  K is symmetric: only the 256 x 256 tiles on or
// above the diagonal are computed (two M = 128 halves in two TMEM accumulators of 256 columns),
// each over a range of 64-row blocks of X (split-K); gram_reduce_kernel sums the ranges in a fixed
// order and writes both triangles, so K is exactly symmetric.  One work item (tile, range) per CTA.
//   warps 0-3  : epilogue: their TMEM lane quarter of both halves -> a column-major partial tile
//                (each store instruction writes 32 consecutive rows of one column)
//   warps 4-11 : converters.  A block of 64 rows arrives as four pieces of 16 rows x 256 float32
//                columns of the tile's row range (A) and column range (B; the same data on the
//                diagonal).  Thread (op, kql, mg) reads rows 8 kql .. 8 kql + 7 of a piece at
//                columns 4 mg .. 4 mg + 3 (16-byte shared loads; eight consecutive threads read one
//                row's consecutive chunks) and writes each column's eight values as one 16-byte
//                bf16 K chunk of a 128-byte-swizzled K-major operand row (the stores meet four-way
//                bank conflicts, which cost less than the selects of a conflict-free store order).
//                Shared-memory traffic per 64-row block (off the diagonal): 128 KB of float32 in by
//                TMA and out to the converters, 64 KB of bf16 operands in, 96 KB read by the MMAs,
//                about 3250 cycles at 128 B / clock against 1170 cycles of MMAs: this kernel is
//                bound by shared-memory bandwidth
//   warp 12    : lane 0 moves the pieces from global memory by TMA into a 3-slot ring
//   warp 13    : TMEM allocation; lane 0 issues tcgen05.mma (M 128, N 256, K 16, both halves) per
//                block and commits each operand stage back to the converters
// Two 64 KB operand stages and three 32 KB pieces: 224 KB of shared memory.  Every wait is
// bounded as in gemm_tc_kernel.
constexpr int GR_TILE = 256, GR_OSTAGES = 2, GR_SLOTS = 3, GR_CONV_WARPS = 8;
constexpr int GR_THREADS = 32 * (4 + GR_CONV_WARPS + 2);
constexpr uint32_t GR_OP_BYTES = GR_TILE * 128;     // one bf16 operand of a stage: 256 rows x 64
constexpr uint32_t GR_STAGE_BYTES = 2 * GR_OP_BYTES;
constexpr uint32_t GR_PIECE_OP = 16 * GR_TILE * 4;  // one operand's float32 piece: 16 rows x 256
constexpr uint32_t GR_SLOT_BYTES = 2 * GR_PIECE_OP;

struct GrParams {
    int64_t n;
    int D, nb, tiles, kbps, nkb;  // nb column blocks of 256, tiles = nb (nb + 1) / 2
    int boxw;                     // float32 columns per TMA row (min(256, D)); row pitch 4 boxw bytes
    float *partial;               // [range][tile][half][column 256][row 128]
    int *status;
};

// upper-triangle tile t (row-major over bi <= bj) -> block row bi, block column bj
__host__ __device__ __forceinline__ void gram_tile(int t, int nb, int &bi, int &bj) {
    bi = 0;
    while (t >= nb - bi) {
        t -= nb - bi;
        ++bi;
    }
    bj = bi + t;
}

__device__ __forceinline__ float f4c(const float4 &v, int j) { return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w; }

__global__ void __launch_bounds__(GR_THREADS, 1)
    gram_f32in_kernel(const __grid_constant__ CUtensorMap tx, const GrParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *slots = base + GR_OSTAGES * GR_STAGE_BYTES;
    uint64_t *ofull = reinterpret_cast<uint64_t *>(slots + GR_SLOTS * GR_SLOT_BYTES);
    uint64_t *oempty = ofull + GR_OSTAGES;
    uint64_t *sfull = oempty + GR_OSTAGES;
    uint64_t *sempty = sfull + GR_SLOTS;
    uint64_t *tfull = sempty + GR_SLOTS;
    uint64_t *drain = tfull + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = (int)blockIdx.x % p.tiles, range = (int)blockIdx.x / p.tiles;
    int bi, bj;
    gram_tile(t, p.nb, bi, bj);
    const bool diag = bi == bj;
    const int kb0 = range * p.kbps, nq = min(p.nkb, kb0 + p.kbps) - kb0;  // >= 1 block
    const int npieces = 4 * nq;
    const int conv = 32 * GR_CONV_WARPS;
    const int W_PROD = 4 + GR_CONV_WARPS, W_MMA = W_PROD + 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < GR_OSTAGES; ++s) {
            mbar_init(ofull + s, conv);
            mbar_init(oempty + s, 1);
        }
        for (int z = 0; z < GR_SLOTS; ++z) {
            mbar_init(sfull + z, 1);
            mbar_init(sempty + z, conv);
        }
        mbar_init(tfull, 1);
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == W_MMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == W_PROD) {
        // ---- TMA producer: piece g = 4 q + pc holds rows 64 (kb0 + q) + 16 pc .. + 15
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)(diag ? 1 : 2) * 16 * p.boxw * 4;
            for (int g = 0; g < npieces; ++g) {
                const int z = g % GR_SLOTS, w = g / GR_SLOTS;
                if (w > 0 && !mbar_wait(sempty + z, (uint32_t)((w - 1) & 1))) {
                    *abort_flag = 1;
                    atomicOr(p.status, ST_TIMEOUT);
                }
                if (*abort_flag) {
                    // drain: the copies already started must land before the CTA exits
                    for (int h = max(0, g - GR_SLOTS); h < g; ++h)
                        mbar_wait(sfull + h % GR_SLOTS, (uint32_t)((h / GR_SLOTS) & 1));
                    break;
                }
                const int row = (kb0 + (g >> 2)) * 64 + 16 * (g & 3);
                uint8_t *dst = slots + (size_t)z * GR_SLOT_BYTES;
                mbar_expect_tx(sfull + z, bytes);
                tma_load_2d(dst, &tx, GR_TILE * bi, row, sfull + z);
                if (!diag) tma_load_2d(dst + GR_PIECE_OP, &tx, GR_TILE * bj, row, sfull + z);
            }
        }
        __syncwarp();
    } else if (warp >= 4 && warp < W_PROD) {
        // ---- converters
        const int ct = threadIdx.x - 128;
        const int mg = ct & 63, kql = (ct >> 6) & 1, op = ct >> 7;
        const bool active = (op == 0 || !diag) && 4 * mg < p.boxw;
        const int pitch = 4 * p.boxw;
        for (int q = 0; q < nq; ++q) {
            const int s = q % GR_OSTAGES;
            uint8_t *dst = base + (size_t)s * GR_STAGE_BYTES + op * GR_OP_BYTES;
            bool ok = !*abort_flag;
            for (int pc = 0; pc < 4 && ok; ++pc) {
                const int g = 4 * q + pc, z = g % GR_SLOTS;
                if (!mbar_wait(sfull + z, (uint32_t)((g / GR_SLOTS) & 1))) {
                    ok = false;
                    break;
                }
                float4 v[8];
                if (active) {
                    const uint8_t *src = slots + (size_t)z * GR_SLOT_BYTES + op * GR_PIECE_OP + 16 * mg;
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        v[i] = *reinterpret_cast<const float4 *>(src + (8 * kql + i) * pitch);
                }
                mbar_arrive(sempty + z);  // the piece is in registers
                if (pc == 0 && q >= GR_OSTAGES && !mbar_wait(oempty + s, (uint32_t)((q / GR_OSTAGES - 1) & 1))) {
                    ok = false;
                    break;
                }
                if (active) {
                    const int kq = 2 * pc + kql;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int row = 4 * mg + j;
                        uint4 o;
                        o.x = pack_bf16x2(f4c(v[0], j), f4c(v[1], j));
                        o.y = pack_bf16x2(f4c(v[2], j), f4c(v[3], j));
                        o.z = pack_bf16x2(f4c(v[4], j), f4c(v[5], j));
                        o.w = pack_bf16x2(f4c(v[6], j), f4c(v[7], j));
                        *reinterpret_cast<uint4 *>(dst + (row >> 3) * 1024 + (row & 7) * 128 + ((kq ^ (row & 7)) << 4)) = o;
                    }
                }
            }
            if (!ok || *abort_flag) {
                *abort_flag = 1;
                atomicOr(p.status, ST_TIMEOUT);
                break;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(ofull + s);
        }
    } else if (warp == W_MMA) {
        // ---- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_tc<0>(TC_BM, GR_TILE);
            bool ok = true;
            for (int q = 0; q < nq; ++q) {
                const int s = q % GR_OSTAGES;
                if (!mbar_wait(ofull + s, (uint32_t)((q / GR_OSTAGES) & 1)) || *abort_flag) {
                    *abort_flag = 1;
                    atomicOr(p.status, ST_TIMEOUT);
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                uint8_t *sa = base + (size_t)s * GR_STAGE_BYTES;
                uint8_t *sb = diag ? sa : sa + GR_OP_BYTES;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint64_t ad = sdesc(sa + h * (GR_OP_BYTES / 2) + 32 * k);
                        const uint64_t bd = sdesc(sb + 32 * k);
                        const uint32_t acc = (q > 0 || k > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\t"
                            "setp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem + (uint32_t)(h * 256)),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                            : "memory");
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(oempty + s))
                             : "memory");
            }
            if (ok)
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(tfull))
                             : "memory");
            // every MMA this thread issued has completed once `drain` flips
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(drain))
                         : "memory");
            if (!mbar_wait(drain, 0)) atomicOr(p.status, ST_TIMEOUT);
        }
        __syncwarp();
    } else {
        // ---- epilogue: TMEM lanes 32 warp .. of both halves -> partial[range][t][half][column][row]
        if (!*abort_flag && mbar_wait(tfull, 0)) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            float *out = p.partial + ((int64_t)range * p.tiles + t) * 2 * GR_TILE * 128;
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
#pragma unroll 1
                for (int c0 = 0; c0 < GR_TILE; c0 += 16) {
                    uint32_t r[16];
                    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(h * 256 + c0), r);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        out[((int64_t)h * GR_TILE + c0 + j) * 128 + warp * 32 + lane] = __uint_as_float(r[j]);
                }
            }
        } else {
            *abort_flag = 1;
            atomicOr(p.status, ST_TIMEOUT);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == W_MMA)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// K from the partial tiles: a block sums one 32 x 32 piece of a tile over the ranges (fixed order),
// writes it transposed (K[j][i], coalesced along i) and, off the diagonal, as is through a shared
// slab (K[i][j], coalesced along j); on a diagonal tile only the pairs i <= j are used, so that
// K[i][j] and K[j][i] are the same float.
__global__ void __launch_bounds__(256) gram_reduce_kernel(const float *__restrict__ part, int ranges, int tiles,
                                                          int nb, int D, float *__restrict__ K) {
    __shared__ float sm[32][33];
    const int t = blockIdx.y;
    int bi, bj;
    gram_tile(t, nb, bi, bj);
    const int R0 = (int)(blockIdx.x >> 3) * 32, C0 = (int)(blockIdx.x & 7) * 32;
    if (bi == bj && R0 > C0) return;  // the mirror block writes these
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int row = R0 + tx, h = row >> 7, rr = row & 127;
    const int64_t I = (int64_t)GR_TILE * bi + row;
    for (int cc = ty; cc < 32; cc += 8) {
        const int col = C0 + cc;
        float acc = 0.f;
        for (int s = 0; s < ranges; ++s)
            acc += part[((((int64_t)s * tiles + t) * 2 + h) * GR_TILE + col) * 128 + rr];
        const int64_t J = (int64_t)GR_TILE * bj + col;
        if (I < D && J < D && (bi < bj || row <= col)) K[J * D + I] = acc;
        sm[cc][tx] = acc;
    }
    __syncthreads();
    for (int a = ty; a < 32; a += 8) {
        const int64_t I2 = (int64_t)GR_TILE * bi + R0 + a, J2 = (int64_t)GR_TILE * bj + C0 + tx;
        if (I2 < D && J2 < D && (bi < bj || R0 + a < C0 + tx)) K[I2 * D + J2] = sm[tx][a];
    }
}

// the float32-input second moment applies: 16-byte aligned rows (D % 4 == 0), at least one 64-row
// block (the TMA box's 16 rows and min(256, D) columns lie inside X)
static bool gram_fused_ok(const float *X, int64_t n, int D) {
    return D % 4 == 0 && ((uintptr_t)X & 15) == 0 && n >= 64 && (n + 63) / 64 < ((int64_t)1 << 31);
}

static int second_moment_f32in(const float *X, int64_t n, int D, float *K, int *status, cudaStream_t st) {
    const int nb = (D + GR_TILE - 1) / GR_TILE, tiles = nb * (nb + 1) / 2;
    const int nkb = (int)((n + 63) / 64);
    const int boxw = std::min(GR_TILE, D);
    CUtensorMap tx;
    {
        // X as float32 pieces of 16 rows x boxw columns (no swizzle); rows >= n and columns >= D
        // read as zeros
        auto fn = encode_fn();
        if (!fn) return fail(LV_ERR_CUDA, "second_moment: cuTensorMapEncodeTiled unavailable");
        cuuint64_t dims[2] = {(cuuint64_t)D, (cuuint64_t)n};
        cuuint64_t strides[1] = {(cuuint64_t)D * 4};
        cuuint32_t box[2] = {(cuuint32_t)boxw, 16};
        cuuint32_t es[2] = {1, 1};
        if (fn(&tx, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(X), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return fail(LV_ERR_CUDA, "second_moment: cuTensorMapEncodeTiled failed for the float32 rows");
    }
    int ranges = std::max(1, std::min(nkb, std::max(1, sm_count()) / tiles));
    const int kbps = (nkb + ranges - 1) / ranges;
    ranges = (nkb + kbps - 1) / kbps;
    float *part = nullptr;
    if (tmp_alloc((void **)&part, sizeof(float) * (size_t)ranges * tiles * 2 * GR_TILE * 128, st))
        return fail(LV_ERR_OOM, "second_moment: allocation failed");
    GrParams p;
    p.n = n;
    p.D = D;
    p.nb = nb;
    p.tiles = tiles;
    p.kbps = kbps;
    p.nkb = nkb;
    p.boxw = boxw;
    p.partial = part;
    p.status = status;
    const size_t sm = (size_t)GR_OSTAGES * GR_STAGE_BYTES + (size_t)GR_SLOTS * GR_SLOT_BYTES + 256 + 1024;
    int rc = LV_OK;
    if (cudaFuncSetAttribute(gram_f32in_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        rc = fail(LV_ERR_CUDA, "second_moment: shared-memory attribute failed");
    if (rc == LV_OK) {
        gram_f32in_kernel<<<(unsigned)(ranges * tiles), GR_THREADS, sm, st>>>(tx, p);
        if (cudaGetLastError() != cudaSuccess) rc = fail(LV_ERR_CUDA, "second_moment: gram_f32in_kernel launch failed");
    }
    if (rc == LV_OK) {
        gram_reduce_kernel<<<dim3(64, (unsigned)tiles), dim3(32, 8), 0, st>>>(part, ranges, tiles, nb, D, K);
        if (cudaGetLastError() != cudaSuccess) rc = fail(LV_ERR_CUDA, "second_moment: gram_reduce_kernel launch failed");
    }
    tmp_free(part, st);
    return rc;
}

int second_moment_bf16(const float *X, int64_t n, int D, float *K, int *status, cudaStream_t st) {
    if (gram_fused_ok(X, n, D)) return second_moment_f32in(X, n, D, K, status, st);
    // otherwise through a transposed bf16 copy of X and the general GEMM
    const int64_t ldt = round_up(n, 8);
    const int tiles = (int)(((D + TC_BM - 1) / TC_BM) * ((D + 255) / 256));
    const int splits = std::max(1, std::min(64, 148 / std::max(1, tiles)));
    __nv_bfloat16 *Xt = nullptr;
    float *work = nullptr;
    int rc = LV_OK;
    if (tmp_alloc((void **)&Xt, (size_t)D * ldt * 2, st) || tmp_alloc((void **)&work, sizeof(float) * (size_t)splits * D * D, st))
        rc = fail(LV_ERR_OOM, "second_moment: allocation failed");
    if (rc == LV_OK) rc = launch_cast_transpose_bf16(X, n, D, Xt, ldt, st);
    if (rc == LV_OK) rc = gemm_bf16_tc(Xt, D, ldt, Xt, D, ldt, n, K, D, splits, work, status, st);
    tmp_free(Xt, st);
    tmp_free(work, st);
    return rc;
}

}  // namespace lv
