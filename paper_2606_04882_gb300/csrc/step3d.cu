// 3D leapfrog step with a shaped stencil (3D extension of Eq.
// spacexz_derivative2_sym as the union of the 2D shape in the three coordinate
// planes), fused with damping, injection, sampling and the FWI modes.
//
// A CTA owns a 64 x TY column of (x, y) and marches a chunk of z planes.  A
// producer warp streams the planes through a ring of shared-memory slots with
// TMA (out-of-bounds zero fill = zero field outside the padded grid), one full
// and one empty mbarrier per slot; the consumer threads (tx, ty) each own 4
// consecutive x (one float4) of row y0 + ty in every plane of the chunk.  Two
// kernels: step3d_cross (z arm in a register queue) and step3d_planar
// (rhombus and square: each plane scattered into a register accumulator of the
// outputs it touches), in step3d_cross.cu and step3d_planar.cu.  This file
// holds the generic kernel for the stencils neither covers, variant selection
// and the launch.
#include "step3d_common.cuh"

namespace fdw {

namespace {

// ---------------------------------------------------------------------------
// Generic 3D kernel: every shape of Section 4.1 (as the union of the 2D shape
// in the three coordinate planes) with any radius 1 <= M <= kMaxM, for the
// stencils no specialised kernel covers.  It gathers the stencil from global
// memory (L1/L2 cached, no staging), with the tile and z-chunk decomposition,
// point tables and modes of the specialised kernels: a CTA walks the 64 x TY
// column of its tile over its z-chunk, thread (tx, ty) owning 4 consecutive x
// of row ty.  Centre-free like the others: every point enters as
// u(x + o) - u(x), grouped by orbit, so a constant field gives exactly zero.
// ---------------------------------------------------------------------------
constexpr int kGenTY = 8;

template <int MODE>
__global__ void __launch_bounds__(16 * kGenTY) step3d_generic(const __grid_constant__ StepParams p,
                                                              int shape, int M, int N)
{
    const int ntile = p.tiles_x * p.tiles_y;
    const int tile = blockIdx.x % ntile, zc = blockIdx.x / ntile;
    const int x0 = (tile % p.tiles_x) * kTX3, y0 = (tile / p.tiles_x) * kGenTY;
    const int zb = zc * p.zchunk;
    const int nz = (int)p.nz, ny = (int)p.ny, nx = (int)p.nx;
    const int ze = min(nz, zb + p.zchunk);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int xg = x0 + 4 * tx, yg = y0 + ty;
    const bool colok = xg < nx && yg < ny;
    const int64_t colo = (int64_t)yg * p.pitch + xg;
    float d2xy[4];
    {
        const float d2y = layer_d2(yg, p.phys_lo[1], p.phys_hi[1]);
#pragma unroll
        for (int j = 0; j < 4; ++j) d2xy[j] = layer_d2(xg + j, p.phys_lo[0], p.phys_hi[0]) + d2y;
    }
    int ki = p.inj_ptr ? p.inj_ptr[tile] : 0, kie = p.inj_ptr ? p.inj_ptr[tile + 1] : 0;
    int ks = p.smp_ptr ? p.smp_ptr[tile] : 0, kse = p.smp_ptr ? p.smp_ptr[tile + 1] : 0;
    int zinj = ki < kie ? p.inj[ki].z : 0x7fffffff;
    int zsmp = ks < kse ? p.smp[ks].z : 0x7fffffff;
    // u at (z, y, x); zero outside the padded grid
    auto at = [&](int z, int y, int x) -> float {
        if ((unsigned)z >= (unsigned)nz || (unsigned)y >= (unsigned)ny || (unsigned)x >= (unsigned)nx) return 0.f;
        return __ldg(p.u_cur + (int64_t)z * p.plane + (int64_t)y * p.pitch + x);
    };
    for (int z = zb; z < ze; ++z) {
        float lap[4] = {0.f, 0.f, 0.f, 0.f}, cc[4] = {0.f, 0.f, 0.f, 0.f};
        if (colok) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int x = xg + j;
                if (x >= nx) continue;
                const float c = at(z, yg, x);
                cc[j] = c;
                float acc = 0.f;
                for (int d = 1; d <= M; ++d) {   // axis orbit (d, 0, 0): six points
                    const float s = ((at(z, yg, x + d) - c) + (at(z, yg, x - d) - c)) +
                                    ((at(z, yg + d, x) - c) + (at(z, yg - d, x) - c)) +
                                    ((at(z + d, yg, x) - c) + (at(z - d, yg, x) - c));
                    acc = fmaf(p.w[d * kWDim], s, acc);
                }
                // off-axis points (a, b), a, b >= 1, of the 2D shape in the xy, xz and yz planes
                for (int b = 1; b <= M; ++b) {
                    const int E = shape_ext(shape, M, N, b);
                    for (int a = 1; a <= E; ++a) {
                        const float w = p.w[max(a, b) * kWDim + min(a, b)];
                        float s = 0.f;
#pragma unroll
                        for (int sa = -1; sa <= 1; sa += 2)
#pragma unroll
                            for (int sb = -1; sb <= 1; sb += 2) {
                                s += (at(z, yg + sb * b, x + sa * a) - c) +      // xy plane
                                     (at(z + sb * b, yg, x + sa * a) - c) +      // xz plane
                                     (at(z + sb * b, yg + sa * a, x) - c);       // yz plane
                            }
                        acc = fmaf(w, s, acc);
                    }
                }
                lap[j] = acc;
            }
        }
        const int64_t off = (int64_t)z * p.plane + colo;
        float4 up = make_float4(0.f, 0.f, 0.f, 0.f), kk = up;
        if (colok) {   // rows are padded to a multiple of 32 floats: the float4 stays in the row
            up = ldg4(p.u_prev + off);
            kk = ldg4(p.kappa + off);
        }
        const float d2z = layer_d2(z, p.phys_lo[2], p.phys_hi[2]);
        const float upa[4] = {up.x, up.y, up.z, up.w}, ka[4] = {kk.x, kk.y, kk.z, kk.w};
        float o[4], dv[4], g[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            g[j] = sponge_g(p.gcoef, d2xy[j] + d2z);
            dv[j] = step_update(cc[j], upa[j], ka[j], lap[j], g[j], o[j]);
        }
        float4 of = make_float4(o[0], o[1], o[2], o[3]);
        if (z >= zinj) {
            const InjOut r = inject_plane<MODE>(p, ki, kie, z, tx, ty, of, kk);
            of = r.o;
            ki = r.k;
            zinj = r.z;
        }
        of.x = sponge_div(of.x, g[0]);
        of.y = sponge_div(of.y, g[1]);
        of.z = sponge_div(of.z, g[2]);
        of.w = sponge_div(of.w, g[3]);
        if (z >= zsmp) {
            const int2 r = sample_plane<MODE>(p, ks, kse, z, tx, ty, of, kk);
            ks = r.x;
            zsmp = r.y;
        }
        if (!colok) continue;
        if (p.check) check_growth(p.status, of);
        *reinterpret_cast<float4 *>(p.u_prev + off) = of;
        if (MODE != kModeAdjoint && p.dseg_out)
            *reinterpret_cast<float4 *>(p.dseg_out + off) = make_float4(dv[0], dv[1], dv[2], dv[3]);
        if (MODE == kModeAdjoint) {
            const float4 dd = ldg4(p.dseg_in + off);
            float4 ga = *reinterpret_cast<float4 *>(p.gacc + off);
            ga.x = fmaf(of.x, dd.x, ga.x); ga.y = fmaf(of.y, dd.y, ga.y);
            ga.z = fmaf(of.z, dd.z, ga.z); ga.w = fmaf(of.w, dd.w, ga.w);
            *reinterpret_cast<float4 *>(p.gacc + off) = ga;
        }
    }
}

// The growth check and the D store are template parameters (the check flag
// and the mode): run-time tests of p.check and p.dseg_out in the store loop
// measured 1-4 % and 1-3 % slower on every step.  The checked instantiation
// runs only on the steps that check (one in kCheckEvery and the last).  The
// three modes share their arithmetic, every operation of which is explicitly
// rounded (nothing the compiler may contract differently in one
// instantiation), so the store-D recompute reproduces the forward sweep bit
// for bit.
KernelFn lookup3(int shape, int M, int ty, int mode, bool check = false)
{
    return shape == FD_CROSS ? lookup_cross3(M, ty, mode, check)
                             : lookup_planar3(shape, M, ty, mode, check);
}

}  // namespace

int select_variant_3d(int shape, int M, int N, int64_t nx, int64_t ny, int64_t nz, Variant *v,
                      int ty_pref)
{
    v->dim = 3;
    v->shape = shape;
    v->M = M;
    v->N = N;
    v->generic = 0;
    const int ty = ty_pref > 0 ? ty_pref : (M <= 4 ? 16 : 8);
    if (!lookup3(shape, M, ty, 0)) {
        // no specialised kernel (or not this tile): the generic kernel
        if (ty_pref > 0 && lookup3(shape, M, M <= 4 ? 16 : 8, 0)) return FD_ERR_UNSUPPORTED;
        if (M < 1 || M > kMaxM) return FD_ERR_UNSUPPORTED;
        v->generic = 1;
        v->tx = kTX3;
        v->tz = kGenTY;
        v->box[0] = kTX3; v->box[1] = kGenTY; v->box[2] = 1;   // maps unused by the kernel
        v->tbox[0] = kTX3; v->tbox[1] = kGenTY;
        v->threads = 16 * kGenTY;
        v->smem = 0;
        return 0;
    }
    v->tx = kTX3;
    v->tz = ty;
    const int HX = round4(M);
    v->box[0] = kTX3 + 2 * HX;
    v->box[1] = ty + 2 * M;
    v->box[2] = 1;
    v->tbox[0] = kTX3;
    v->tbox[1] = ty;
    {   // warp-specialised pipelines (cross and planar): one extra producer warp
        const int A = ((kTX3 + 2 * HX) * (ty + 2 * M) + 31) & ~31;
        v->smem = (size_t)ring_depth(A + 3 * kTX3 * ty, ctas_per_sm(shape == FD_CROSS, M, ty)) *
                  (A + 3 * kTX3 * ty) * sizeof(float);
        v->threads = 16 * ty + 32;
    }
    (void)nx; (void)ny; (void)nz;
    return 0;
}

int variants_3d(int shape, int M, int *ty_out, int cap)
{
    int n = 0;
    for (int ty : {16, 8})
        if (n < cap && lookup3(shape, M, ty, 0)) ty_out[n++] = ty;
    return n;
}

// Resident CTAs per SM of a 3D variant's kernel (registers, shared memory and
// threads all counted), 0 on error.
int occupancy_3d(const Variant &v)
{
    if (v.generic) {
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, step3d_generic<kModeForward>, v.threads, 0) !=
            cudaSuccess)
            return 0;
        return per;
    }
    KernelFn fn = lookup3(v.shape, v.M, v.tz, kModeForward);
    if (!fn) return 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem) != cudaSuccess)
        return 0;
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, v.threads, v.smem) != cudaSuccess) return 0;
    return per;
}

cudaError_t launch_step3d(const Variant &v, int mode, const StepParams &p, cudaStream_t s)
{
    if (v.generic) {
        void (*gfn)(const StepParams, int, int, int) =
            mode == kModeAdjoint ? step3d_generic<kModeAdjoint> : step3d_generic<kModeForward>;
        const int grid = p.tiles_x * p.tiles_y * p.nz_chunks;
        if (grid <= 0) return cudaSuccess;
        gfn<<<grid, v.threads, 0, s>>>(p, v.shape, v.M, v.N);
        return cudaGetLastError();
    }
    KernelFn fn = lookup3(v.shape, v.M, v.tz, mode, p.check != 0);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e =
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
    if (e != cudaSuccess) return e;
    const int grid = p.tiles_x * p.tiles_y * p.nz_chunks;
    if (grid <= 0) return cudaSuccess;
    fn<<<grid, v.threads, v.smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace fdw
