/*
 * lb_store.cuh -- population storage formats and their vector loads / stores.
 *
 * The kernels work on the deviation d = f / w_alpha - rho0 of a population from the
 * rest state w_alpha rho0 (all arithmetic is cancellation-free in d: the stencil is
 * linear and minmod is positively homogeneous, so scaling by 1 / w_alpha commutes with
 * the TVD flux). LB_STORE_F64 / LB_STORE_F32 hold f itself, the *_DEV forms hold d.
 */
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

namespace lbk {

template <int ST>
struct Store;

template <>
struct Store<0> {   /* LB_STORE_F64 */
    using T = double;
    using R = double;
    static constexpr bool dev = false;
};
template <>
struct Store<1> {   /* LB_STORE_F32 */
    using T = float;
    using R = float;
    static constexpr bool dev = false;
};
template <>
struct Store<2> {   /* LB_STORE_F32_DEV */
    using T = float;
    using R = float;
    static constexpr bool dev = true;
};
template <>
struct Store<3> {   /* LB_STORE_F16_DEV */
    using T = __half;
    using R = float;
    static constexpr bool dev = true;
};
template <>
struct Store<4> {   /* LB_STORE_BF16_DEV */
    using T = __nv_bfloat16;
    using R = float;
    static constexpr bool dev = true;
};

__device__ __forceinline__ float to_r(float v) { return v; }
__device__ __forceinline__ double to_r(double v) { return v; }
__device__ __forceinline__ float to_r(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_r(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T, typename R>
__device__ __forceinline__ T from_r(R v);
template <>
__device__ __forceinline__ double from_r<double, double>(double v) { return v; }
template <>
__device__ __forceinline__ float from_r<float, float>(float v) { return v; }
template <>
__device__ __forceinline__ __half from_r<__half, float>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_r<__nv_bfloat16, float>(float v) { return __float2bfloat16_rn(v); }

/* stored value -> deviation */
template <int ST>
__device__ __forceinline__ typename Store<ST>::R decode(typename Store<ST>::T v, typename Store<ST>::R winv,
                                                       typename Store<ST>::R rho0)
{
    using R = typename Store<ST>::R;
    if constexpr (Store<ST>::dev) {
        return to_r(v);
    } else {
        return fma(to_r(v), winv, -rho0);
    }
    return R(0);
}

/* deviation -> stored value */
template <int ST>
__device__ __forceinline__ typename Store<ST>::T encode(typename Store<ST>::R d, typename Store<ST>::R w,
                                                       typename Store<ST>::R rho0)
{
    using T = typename Store<ST>::T;
    if constexpr (Store<ST>::dev) {
        return from_r<T>(d);
    } else {
        return from_r<T>(w * (rho0 + d));
    }
}

/* Per-column reference density (deviation formats only): the stored value is
 * d - delta with delta = rho0(x) - rho0 of the node's column, so that a lattice whose
 * density varies along x keeps small stored magnitudes. The arithmetic frame (d) is
 * the same as without it. */
template <int ST>
__device__ __forceinline__ typename Store<ST>::R decode_col(typename Store<ST>::T v, typename Store<ST>::R winv,
                                                           typename Store<ST>::R rho0, typename Store<ST>::R delta)
{
    if constexpr (Store<ST>::dev) return to_r(v) + delta;
    else return decode<ST>(v, winv, rho0);
}
template <int ST>
__device__ __forceinline__ typename Store<ST>::T encode_col(typename Store<ST>::R d, typename Store<ST>::R w,
                                                           typename Store<ST>::R rho0, typename Store<ST>::R delta)
{
    if constexpr (Store<ST>::dev) return encode<ST>(d - delta, w, rho0);
    else return encode<ST>(d, w, rho0);
}

/* ---- stochastic rounding of the 16-bit deviation formats ----
 * A per-step increment below half a unit in the last place of the stored deviation is
 * lost by round-to-nearest every step, and the state stagnates away from the solution.
 * Rounding up or down with the probabilities that make the expected stored value equal
 * the exact one keeps those increments on average. The random bits come from a
 * counter-based generator: C. Wellons' "lowbias32" integer hash (xorshift-multiply
 * finaliser, published 2018) of a key naming the node, the population and the step, so
 * every kernel layout draws the same bits for the same store. */
__device__ __forceinline__ uint32_t lowbias32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

__device__ __forceinline__ uint32_t sr_bits(int x, int j, int nx, int a, uint32_t step)
{
    return lowbias32(lowbias32((uint32_t)j * (uint32_t)nx + (uint32_t)x) ^ lowbias32(((uint32_t)a << 24) ^ step));
}

/* BF16 is the upper half of FP32: adding 16 random bits below the kept half and
 * truncating carries into it with probability equal to the dropped fraction (of the
 * magnitude: the pattern is sign-magnitude). */
__device__ __forceinline__ __nv_bfloat16 sr_bf16(float v, uint32_t r)
{
    uint32_t b = __float_as_uint(v);
    if ((b & 0x7f800000u) == 0x7f800000u) return __float2bfloat16_rn(v);   /* inf, nan */
    b += r & 0xffffu;
    __nv_bfloat16_raw raw;
    raw.x = (unsigned short)(b >> 16);
    return __nv_bfloat16(raw);
}

/* FP16: the neighbour toward zero and the next code away from zero bracket v; the
 * latter is taken with probability (v - lo) / (hi - lo). */
__device__ __forceinline__ __half sr_half(float v, uint32_t r)
{
    const __half lo = __float2half_rz(v);
    const float lof = __half2float(lo);
    if (!(fabsf(v) < 65504.0f) || lof == v) return __float2half_rn(v);
    const __half hi = __ushort_as_half((unsigned short)(__half_as_ushort(lo) + 1u));
    const float frac = (v - lof) / (__half2float(hi) - lof);
    const float u = (float)(r >> 8) * (1.0f / 16777216.0f);
    return u < frac ? hi : lo;
}

/* deviation -> stored value, stochastically rounded for the 16-bit formats (r: random
 * bits), as encode() otherwise */
template <int ST>
__device__ __forceinline__ typename Store<ST>::T encode_sr(typename Store<ST>::R d, typename Store<ST>::R w,
                                                          typename Store<ST>::R rho0, uint32_t r)
{
    if constexpr (ST == 3) return sr_half(d, r);
    else if constexpr (ST == 4) return sr_bf16(d, r);
    else return encode<ST>(d, w, rho0);
}

/* Four consecutive elements (16-byte aligned for FP32, 32 for FP64, 8 for 16-bit). */
template <typename T>
__device__ __forceinline__ void ld4(const T *p, T v[4]);
template <>
__device__ __forceinline__ void ld4<float>(const float *p, float v[4])
{
    float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
template <>
__device__ __forceinline__ void ld4<double>(const double *p, double v[4])
{
    double2 a = reinterpret_cast<const double2 *>(p)[0];
    double2 b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
template <>
__device__ __forceinline__ void ld4<__half>(const __half *p, __half v[4])
{
    uint2 q = *reinterpret_cast<const uint2 *>(p);
    __half2 a = *reinterpret_cast<__half2 *>(&q.x), b = *reinterpret_cast<__half2 *>(&q.y);
    v[0] = __low2half(a); v[1] = __high2half(a); v[2] = __low2half(b); v[3] = __high2half(b);
}
template <>
__device__ __forceinline__ void ld4<__nv_bfloat16>(const __nv_bfloat16 *p, __nv_bfloat16 v[4])
{
    uint2 q = *reinterpret_cast<const uint2 *>(p);
    __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162 *>(&q.x), b = *reinterpret_cast<__nv_bfloat162 *>(&q.y);
    v[0] = __low2bfloat16(a); v[1] = __high2bfloat16(a); v[2] = __low2bfloat16(b); v[3] = __high2bfloat16(b);
}

/* Two consecutive elements (8-byte aligned for FP32, 16 for FP64, 4 for 16-bit). */
template <typename T>
__device__ __forceinline__ void ld2(const T *p, T v[2]);
template <>
__device__ __forceinline__ void ld2<float>(const float *p, float v[2])
{
    float2 q = *reinterpret_cast<const float2 *>(p);
    v[0] = q.x; v[1] = q.y;
}
template <>
__device__ __forceinline__ void ld2<double>(const double *p, double v[2])
{
    double2 q = *reinterpret_cast<const double2 *>(p);
    v[0] = q.x; v[1] = q.y;
}
template <>
__device__ __forceinline__ void ld2<__half>(const __half *p, __half v[2])
{
    __half2 q = *reinterpret_cast<const __half2 *>(p);
    v[0] = __low2half(q); v[1] = __high2half(q);
}
template <>
__device__ __forceinline__ void ld2<__nv_bfloat16>(const __nv_bfloat16 *p, __nv_bfloat16 v[2])
{
    __nv_bfloat162 q = *reinterpret_cast<const __nv_bfloat162 *>(p);
    v[0] = __low2bfloat16(q); v[1] = __high2bfloat16(q);
}

template <typename T>
__device__ __forceinline__ void st4(T *p, const T v[4]);
template <>
__device__ __forceinline__ void st4<float>(float *p, const float v[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void st4<double>(double *p, const double v[4])
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}
template <>
__device__ __forceinline__ void st4<__half>(__half *p, const __half v[4])
{
    __half2 a = __halves2half2(v[0], v[1]), b = __halves2half2(v[2], v[3]);
    uint2 q;
    q.x = *reinterpret_cast<uint32_t *>(&a);
    q.y = *reinterpret_cast<uint32_t *>(&b);
    *reinterpret_cast<uint2 *>(p) = q;
}
template <>
__device__ __forceinline__ void st4<__nv_bfloat16>(__nv_bfloat16 *p, const __nv_bfloat16 v[4])
{
    __nv_bfloat162 a = __halves2bfloat162(v[0], v[1]), b = __halves2bfloat162(v[2], v[3]);
    uint2 q;
    q.x = *reinterpret_cast<uint32_t *>(&a);
    q.y = *reinterpret_cast<uint32_t *>(&b);
    *reinterpret_cast<uint2 *>(p) = q;
}

template <typename T>
__device__ __forceinline__ void st2(T *p, const T v[2]);
template <>
__device__ __forceinline__ void st2<float>(float *p, const float v[2])
{
    *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
}
template <>
__device__ __forceinline__ void st2<double>(double *p, const double v[2])
{
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
}
template <>
__device__ __forceinline__ void st2<__half>(__half *p, const __half v[2])
{
    *reinterpret_cast<__half2 *>(p) = __halves2half2(v[0], v[1]);
}
template <>
__device__ __forceinline__ void st2<__nv_bfloat16>(__nv_bfloat16 *p, const __nv_bfloat16 v[2])
{
    *reinterpret_cast<__nv_bfloat162 *>(p) = __halves2bfloat162(v[0], v[1]);
}

/* N = 2 or 4 consecutive elements (alignment as ld2 / ld4) */
template <int N, typename T>
__device__ __forceinline__ void ldn(const T *p, T v[N])
{
    if constexpr (N == 4) ld4(p, v);
    else ld2(p, v);
}
template <int N, typename T>
__device__ __forceinline__ void stn(T *p, const T v[N])
{
    if constexpr (N == 4) st4(p, v);
    else st2(p, v);
}

/* minmod(a, b) = median(a, b, 0): the smaller-magnitude slope when both have one sign,
 * else 0 (the Sec. 3.1 limiter Psi(Theta) times the difference it multiplies). */
__device__ __forceinline__ float minmod(float a, float b) { return fmaxf(fminf(a, b), fminf(fmaxf(a, b), 0.0f)); }
__device__ __forceinline__ double minmod(double a, double b) { return fmax(fmin(a, b), fmin(fmax(a, b), 0.0)); }

/* The same median written as max(min(a, b), min(a, 0), min(b, 0)), with the
 * negative parts an = min(a, 0), bn = min(b, 0) supplied by the caller: along a row of
 * differences each one serves two neighbouring faces, so its negative part is formed
 * once. FP32 uses the three-input max of sm_100+. */
__device__ __forceinline__ float neg_part(float a) { return fminf(a, 0.0f); }
__device__ __forceinline__ double neg_part(double a) { return fmin(a, 0.0); }
__device__ __forceinline__ float minmod_n(float a, float b, float an, float bn)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(fminf(a, b)), "f"(an), "f"(bn));
    return r;
}
__device__ __forceinline__ double minmod_n(double a, double b, double an, double bn)
{
    return fmax(fmin(a, b), fmax(an, bn));
}

}  // namespace lbk
