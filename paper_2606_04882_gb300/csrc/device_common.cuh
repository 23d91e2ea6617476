// Device helpers: shape geometry, shared-memory barriers and TMA copies
// (inline PTX, sm_100-family), bounded waits, damping.
#pragma once

#include <cstdint>

#include "internal.h"

namespace fdw {

// ---------------------------------------------------------------------------
// Stencil geometry (Section 4.1).  ext(q) = largest |p| of a point (p, q) of
// the 2D shape on row offset |q| (-1: no point besides none; the axis point
// (0, q) always exists for q <= M).  3D shapes are the union of the 2D shape
// in the three coordinate planes, so the same function drives them.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int shape_ext(int shape, int M, int N, int q)
{
    return q == 0 ? M
         : q > M ? -1
         : shape == FD_CROSS ? 0
         : shape == FD_RHOMBUS ? M - q
         : shape == FD_SQUARE ? M
         : shape == FD_CROSS_RHOMBUS ? (q < N ? N - q : 0)
         : /* FD_CROSS_SQUARE */ (q <= N ? M : N);
}

__host__ __device__ constexpr int round4(int x) { return (x + 3) & ~3; }

// ---------------------------------------------------------------------------
// mbarrier + TMA (PTX ISA 8.x, sm_90+; used here on sm_103a)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Expect `bytes` more transaction bytes in the current phase (no arrival).
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait with a time bound of about `cycles` SM clocks; false on time-out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  long long cycles = kWaitCycles)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > cycles) return false;
        __nanosleep(64);
    }
}

// 2D tile load: box at (x, y) of the map into dst; completes on `bar`.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// 3D tile load: box at (x, y, z).
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Growth check of a step's outputs: a value that is non-finite or above
// kBlowupAmp in magnitude marks the run unstable (the comparison is false for
// NaN, so NaN is caught too).
__device__ __forceinline__ void check_growth(int *status, const float4 &o)
{
    if (!(fabsf(o.x) <= kBlowupAmp && fabsf(o.y) <= kBlowupAmp && fabsf(o.z) <= kBlowupAmp &&
          fabsf(o.w) <= kBlowupAmp))
        atomicOr(status, kStatusBlowup);
}

// ---------------------------------------------------------------------------
// Damping: squared node distance into the sponge along one axis.
// ---------------------------------------------------------------------------
// (32-bit integer arithmetic: padded sizes are below 2^24 per axis, and a
// 64-bit integer to float conversion would run on the FP64 pipe.)
__device__ __forceinline__ float layer_d2(int64_t i, int64_t lo, int64_t hi)
{
    const int ii = (int)i, l = (int)lo, h = (int)hi;
    const int d = ii < l ? l - ii : (ii > h ? ii - h : 0);
    return __int2float_rn(d * d);
}

// Leapfrog bracket o = 2u - (1-g)u_prev + kappa lap, written as
//   o = u + (kappa*lap + (g*u_prev + (u - u_prev)))
// with explicit roundings and fused multiply-adds: the increment is formed at
// its own (small) scale and meets u in one rounding, where ((u - u_prev) + u)
// + kappa*lap rounds twice at the scale of u; over a long run that halves the
// dominant rounding error.  Nothing is left for the code generator to contract,
// so every kernel mode (forward, store-D, adjoint) rounds identically.
// Returns D = kappa * lap (its own rounded product).
__device__ __forceinline__ float step_update(float u, float up, float k, float lap, float g,
                                             float &o)
{
    o = __fadd_rn(u, fmaf(k, lap, fmaf(g, up, __fsub_rn(u, up))));
    return __fmul_rn(k, lap);
}

// ---------------------------------------------------------------------------
// Packed FP32x2 arithmetic (sm_100 family): one instruction for two lanes,
// each lane rounded exactly like the scalar operation.
// ---------------------------------------------------------------------------
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk2(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk2(f32x2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
// float4 in shared memory as two packed pairs (x, y) and (z, w)
// (w[i] + w[j], w[i+1] + w[j+1]) for a window w held in registers (i, j
// compile-time after unrolling): one packed add when both pairs start on an
// even element (an aligned register pair of the float4 they were loaded as),
// else two scalar adds whose results the compiler places as a pair, instead of
// moving misaligned operands into pairs first.  The same IEEE adds either way.
__device__ __forceinline__ f32x2 pair_add(const float *w, int i, int j)
{
    if (((i | j) & 1) == 0) return add2(pk2(w[i], w[i + 1]), pk2(w[j], w[j + 1]));
    return pk2(w[i] + w[j], w[i + 1] + w[j + 1]);
}

__device__ __forceinline__ void ld4x2(const float *p, f32x2 &a, f32x2 &b)
{
    const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(p);
    a = v.x;
    b = v.y;
}
// Packed form of step_update (the same roundings, lane by lane).  The fused
// multiply-adds are written out because a packed multiply whose only use is a
// packed add may be fused by the code generator: a bracket written as separate
// multiplies and adds would round differently in a kernel that also stores D
// (a second use of the product) than in one that does not.
__device__ __forceinline__ f32x2 step_update2(f32x2 u, f32x2 up, f32x2 k, f32x2 lap, f32x2 g,
                                              f32x2 &o)
{
    o = add2(u, fma2(k, lap, fma2(g, up, sub2(u, up))));
    return mul2(k, lap);
}

__device__ __forceinline__ float4 ld4(const float *p)
{
    return *reinterpret_cast<const float4 *>(p);
}

__device__ __forceinline__ float4 ldg4(const float *p)
{
    return __ldg(reinterpret_cast<const float4 *>(p));
}

__device__ __forceinline__ float get4(const float4 &v, int j)
{
    return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}

// The scalar parts of the step (the sponge factor and division, the source
// term added inside the bracket) use explicit rounding too, so that no
// instantiation of a step kernel (mode, growth check) can contract them
// differently from another: g = gcoef * d2, o / (1 + g), scale * series.
__device__ __forceinline__ float sponge_g(float gcoef, float d2)
{
    return __fmul_rn(gcoef, d2);
}

__device__ __forceinline__ float sponge_div(float o, float g)
{
    return g != 0.f ? __fdividef(o, __fadd_rn(1.f, g)) : o;
}

__device__ __forceinline__ float src_term(float scale, float series)
{
    return __fmul_rn(scale, series);
}

__device__ __forceinline__ void add4(float4 &v, int j, float a)
{
    v.x = __fadd_rn(v.x, (j == 0) ? a : 0.f);
    v.y = __fadd_rn(v.y, (j == 1) ? a : 0.f);
    v.z = __fadd_rn(v.z, (j == 2) ? a : 0.f);
    v.w = __fadd_rn(v.w, (j == 3) ? a : 0.f);
}

}  // namespace fdw
