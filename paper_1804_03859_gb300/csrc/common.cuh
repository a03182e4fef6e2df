// Shared device/host helpers of the nsstab library: complex arithmetic on
// the CUDA vector types, error plumbing for the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/nsstab.h"
#include "df64.cuh"

namespace nsstab {

// ------------------------------------------------------------ complex types
template <class T> struct cx_t;
template <> struct cx_t<double> { using type = double2; };
template <> struct cx_t<float> { using type = float2; };
template <> struct cx_t<df64> { using type = df64c; };
template <class T> using Cx = typename cx_t<T>::type;

template <class T> __host__ __device__ __forceinline__ Cx<T> mk(T x, T y) {
    Cx<T> r;
    r.x = x;
    r.y = y;
    return r;
}
template <class C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <class C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <class C> __device__ __forceinline__ C cconj(C a) { C r; r.x = a.x; r.y = -a.y; return r; }
// a * b
template <class C> __device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// a * conj(b)
template <class C> __device__ __forceinline__ C cmulc(C a, C b) {
    C r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.y * b.x - a.x * b.y;
    return r;
}
template <class C, class T> __device__ __forceinline__ C cscale(C a, T s) { C r; r.x = a.x * s; r.y = a.y * s; return r; }
// multiply by -i and by +i
template <class C> __device__ __forceinline__ C cmul_mi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }
template <class C> __device__ __forceinline__ C cmul_pi(C a) { C r; r.x = -a.y; r.y = a.x; return r; }

// two adjacent complex values as one access (16 B for float, two 16-B
// halves of one 32-B sector for double)
template <class T> struct PairIO;
template <> struct PairIO<float> {
    __device__ static __forceinline__ void load(const float2* p, float2& a, float2& b) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        a.x = v.x; a.y = v.y; b.x = v.z; b.y = v.w;
    }
    __device__ static __forceinline__ void store(float2* p, float2 a, float2 b) {
        *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
    }
};
template <> struct PairIO<double> {
    __device__ static __forceinline__ void load(const double2* p, double2& a, double2& b) {
        a = p[0];
        b = p[1];
    }
    __device__ static __forceinline__ void store(double2* p, double2 a, double2 b) {
        p[0] = a;
        p[1] = b;
    }
};

template <> struct PairIO<df64> {
    __device__ static __forceinline__ void load(const df64c* p, df64c& a, df64c& b) {
        a = p[0];
        b = p[1];
    }
    __device__ static __forceinline__ void store(df64c* p, df64c a, df64c b) {
        p[0] = a;
        p[1] = b;
    }
};

// read-only cached load of one complex value
__device__ __forceinline__ float2 ldg_c(const float2* p) { return __ldg(p); }
__device__ __forceinline__ double2 ldg_c(const double2* p) { return __ldg(p); }
__device__ __forceinline__ df64c ldg_c(const df64c* p) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    df64c r;
    r.x = df64(v.x, v.y);
    r.y = df64(v.z, v.w);
    return r;
}

// --------------------------------------------------------------- errors
void set_error(const std::string& msg);
const char* last_error();

#define NS_CUDA(call)                                                            \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            ::nsstab::set_error(std::string(#call) + ": " + cudaGetErrorString(e_)); \
            return e_ == cudaErrorMemoryAllocation ? NSSTAB_ERR_OUT_OF_MEMORY    \
                                                   : NSSTAB_ERR_CUDA;            \
        }                                                                        \
    } while (0)

#define NS_LAUNCH_CHECK()                                                        \
    do {                                                                         \
        cudaError_t e_ = cudaGetLastError();                                     \
        if (e_ != cudaSuccess) {                                                 \
            ::nsstab::set_error(std::string("kernel launch: ") + cudaGetErrorString(e_)); \
            return NSSTAB_ERR_CUDA;                                              \
        }                                                                        \
    } while (0)

#define NS_TRY(expr)                  \
    do {                              \
        int rc_ = (expr);             \
        if (rc_ < 0) return rc_;      \
    } while (0)

inline bool is_pow2(long v) { return v > 0 && (v & (v - 1)) == 0; }
inline int ilog2(long v) {
    int r = 0;
    while ((1L << r) < v) ++r;
    return r;
}

}  // namespace nsstab
