// Device helpers of the 3D step kernels: residency and ring depth, the
// per-tile point-table walk, and the out-of-line injection and sampling of the
// planes that carry table entries.
#pragma once

#include "device_common.cuh"

namespace fdw {

namespace {

constexpr int kTX3 = 64;

// CTAs per SM the warp-specialised pipelines are built for: 2 with 64 x 16
// tiles; with 64 x 8 tiles 4 for the cross up to M = 4 (96 registers per
// thread suffice) and 3 otherwise (the planar kernels run faster with the
// registers of 3).
__host__ __device__ constexpr int ctas_per_sm(bool cross, int M, int ty)
{
    return ty >= 16 ? 2 : (cross && M <= 4 ? 4 : 3);
}

// Ring depth: as many plane slots (4 to 8) as fit the shared memory of one
// CTA at that residency; deeper rings keep more planes of copies in flight.
__host__ __device__ constexpr int ring_depth(int slot_floats, int ctas)
{
    const int budget = (ctas <= 2 ? 80 : ctas == 3 ? 72 : 54) * 1024;
    const int n = budget / (slot_floats * 4);
    return n < 4 ? 4 : n > 8 ? 8 : n;
}

// Tile table walk for one plane: apply f(j, entry) to this thread's entries
// with entry.z == z.  Entries are sorted by (z, y, x) within a tile, so the
// plane's segment and, inside it, this thread's row and 4 columns are found
// by binary search; `k` advances to the first entry of a later plane.
__device__ __forceinline__ long long entry_key(int z, int yx)
{
    return ((long long)z << 32) | (unsigned)yx;
}

__device__ __forceinline__ int first_at_least(const PtEntry *tab, int lo, int hi, long long key)
{
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (entry_key(tab[mid].z, tab[mid].yx) < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <class F>
__device__ __forceinline__ void plane_entries(const PtEntry *tab, int &k, int kend, int z,
                                              int tx, int ty, F f)
{
    const int zb = first_at_least(tab, k, kend, entry_key(z, 0));
    const int ze = first_at_least(tab, zb, kend, entry_key(z + 1, 0));
    const int lo = (ty << 16) | (4 * tx), hi = lo + 4;
    for (int i = first_at_least(tab, zb, ze, entry_key(z, lo)); i < ze; ++i) {
        const PtEntry en = tab[i];
        if (en.yx >= hi) break;
        f(en.yx & 3, en);
    }
    k = ze;
}

// Out-of-line handlers for the (rare) planes that carry table entries, so the
// unrolled plane loops stay small.  Everything goes in and out by value (a
// reference would force the caller's registers into local memory every
// plane); they return the next pending entry and its z.
struct InjOut {
    float4 o;
    int k, z;
};

template <int MODE>
__device__ __noinline__ InjOut inject_plane(const StepParams &p, int k, int kend, int z, int tx,
                                            int ty, float4 o, float4 kk)
{
    plane_entries(p.inj, k, kend, z, tx, ty, [&](int j, const PtEntry &en) {
        float a = src_term(en.scale, p.inj_series[(int64_t)p.step * p.inj_ncol + en.col]);
        if (MODE == kModeAdjoint) a = __fmul_rn(a, get4(kk, j));
        add4(o, j, a);
    });
    InjOut r;
    r.o = o;
    r.k = k;
    r.z = k < kend ? p.inj[k].z : 0x7fffffff;
    return r;
}

template <int MODE>
__device__ __noinline__ int2 sample_plane(const StepParams &p, int k, int kend, int z, int tx,
                                          int ty, float4 o, float4 kk)
{
    plane_entries(p.smp, k, kend, z, tx, ty, [&](int j, const PtEntry &en) {
        float v = get4(o, j) * en.scale;
        if (MODE == kModeAdjoint) v /= get4(kk, j);
        p.smp_out[(int64_t)p.step * p.smp_ncol + en.col] = v;
    });
    return make_int2(k, k < kend ? p.smp[k].z : 0x7fffffff);
}

using KernelFn = void (*)(const StepParams);

}  // namespace

// Instantiation lookups of the specialised kernels (step3d_cross.cu,
// step3d_planar.cu): the kernel for a shape, radius, tile row count, mode and
// growth check, or nullptr where none is built.
KernelFn lookup_cross3(int M, int ty, int mode, bool check);
KernelFn lookup_planar3(int shape, int M, int ty, int mode, bool check);

}  // namespace fdw
