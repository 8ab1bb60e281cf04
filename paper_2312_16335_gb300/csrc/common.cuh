// Shared device/host helpers for the LeanVec CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>

#include "../../include/leanvec.h"

namespace lv {

constexpr unsigned FULL = 0xffffffffu;
constexpr int RMAX = 128;        // largest supported graph out-degree
constexpr int LCAP_MAX = 512;    // largest supported beam
constexpr uint32_t EXPANDED = 0x80000000u;

// device status bits (OR-ed into the per-index status word)
constexpr int ST_CAPACITY = 1;
constexpr int ST_CORRUPT = 2;
constexpr int ST_TIMEOUT = 4;

void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

// scratch memory from the library's stream-ordered pool (pool.cu)
int tmp_alloc(void **p, size_t bytes, cudaStream_t st);
void tmp_free(void *p, cudaStream_t st);

#define LV_CUDA(call)                                              \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return ::lv::cuda_fail(_e, #call);  \
    } while (0)

#define LV_CHECK_LAUNCH(what)                                      \
    do {                                                           \
        cudaError_t _e = cudaGetLastError();                       \
        if (_e != cudaSuccess) return ::lv::cuda_fail(_e, what);   \
    } while (0)

inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// Record geometry of an LVQ / float32 record (see leanvec.h).  LVQ records of an L2 index carry a
// second 16-byte constants chunk {N, ||x||^2, 0, 0} after {delta, lower, G, H}.
struct RecGeom {
    int dim = 0, bits = 0;
    int code_bytes = 0;   // zero-padded code area (multiple of 16)
    int code_chunks = 0;  // code_bytes / 16
    int64_t stride = 0;
};

inline bool rec_geom(int dim, int bits, RecGeom &g, int metric = 0) {
    if (dim <= 0) return false;
    g.dim = dim;
    g.bits = bits;
    if (bits == 8 || bits == 4) {
        int cb = bits == 8 ? dim : (dim + 1) / 2;
        g.code_bytes = (int)round_up(cb, 16);
        g.code_chunks = g.code_bytes / 16;
        g.stride = round_up(g.code_bytes + (metric ? 32 : 16), 32);
        return true;
    }
    if (bits == 16) {  // IEEE half vectors, no constants
        g.code_bytes = (int)round_up((int64_t)dim * 2, 16);
        g.code_chunks = g.code_bytes / 16;
        g.stride = round_up((int64_t)dim * 2, 32);
        return true;
    }
    if (bits == 32) {
        g.code_bytes = (int)round_up((int64_t)dim * 4, 16);
        g.code_chunks = g.code_bytes / 16;
        g.stride = round_up((int64_t)dim * 4, 32);
        return true;
    }
    return false;
}

// ---------------------------------------------------------------- device side
__device__ __forceinline__ uint4 ldg_stream(const void *p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// float(b) for the byte of w selected by SEL, exact: builds 2^23 + b and subtracts 2^23.
template <int SEL>
__device__ __forceinline__ float byte_to_float(uint32_t w) {
    uint32_t bits = __byte_perm(w, 0x4B000000u, 0x7540u | SEL);
    return __int_as_float((int)bits) - 8388608.0f;
}

// The exact build score <y_a, y_b> of two primaries (see leanvec.h): integer sums P and the
// per-record terms combined by one fixed sequence of float32 operations (no FMA).
__device__ __forceinline__ float build_pair_score(float mu2, float fdim, float da, float la, float Ga, float Ha,
                                                  float db, float lb, float Gb, float Hb, int P) {
    float t1 = __fadd_rn(Ga, Gb);
    float t2 = __fmul_rn(fdim, __fmul_rn(la, lb));
    float t3 = __fadd_rn(__fmul_rn(lb, Ha), __fmul_rn(la, Hb));
    float t4 = __fmul_rn(__fmul_rn(da, db), __int2float_rn(P));
    float s = __fadd_rn(mu2, t1);
    s = __fadd_rn(s, t2);
    s = __fadd_rn(s, t3);
    return __fadd_rn(s, t4);
}

// L2 build score -||y_a - y_b||^2 = 2 <y_a, y_b> - (N_a + N_b), N = self scores (symmetric)
__device__ __forceinline__ float l2_from_ip(float ip, float Na, float Nb) {
    return __fsub_rn(__fmul_rn(2.0f, ip), __fadd_rn(Na, Nb));
}

__device__ __forceinline__ bool key_better(float sa, int ia, float sb, int ib) {
    return sa > sb || (sa == sb && ia < ib);
}

}  // namespace lv
