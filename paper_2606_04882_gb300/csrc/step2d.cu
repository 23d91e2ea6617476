// 2D leapfrog step with a shaped stencil (paper Eq. spacexz_derivative2_sym,
// Eq. time_derivative1, damping term of Section 3.1), fused with point-source
// injection, receiver sampling and the FWI modes (store D / adjoint with
// gradient accumulation).
//
// One CTA computes a tile of 64 columns x (16 R) rows.  The tile plus its halo
// (HX = round4(M) columns, M rows on each side) is brought into shared memory
// by one TMA load whose out-of-bounds elements are zero-filled: that is the
// zero field outside the padded grid.  Thread (tx, ty) owns 4 consecutive
// columns (one float4) of R consecutive rows.
#include <algorithm>

#include "device_common.cuh"

namespace fdw {

namespace {

constexpr int kTX = 64;     // output columns per tile
constexpr int kTZ = 16;     // thread rows per tile
constexpr int kThreads = 256;

// Point tables hold each tile's entries sorted by (z, x): the entries of row
// zg and thread column tx (x in [4 tx, 4 tx + 4)) are found by binary search
// in [b, e) and f(j, entry) is applied to each, j = x - 4 tx.
__device__ __forceinline__ long long entry_key(int z, int x)
{
    return ((long long)z << 32) | (unsigned)x;
}

template <class F>
__device__ __forceinline__ void for_row(const PtEntry *tab, int b, int e, int zg, int tx, F f)
{
    const long long lo = entry_key(zg, 4 * tx), hi = entry_key(zg, 4 * tx + 4);
    int l = b, h = e;
    while (l < h) {
        const int mid = (l + h) >> 1;
        if (entry_key(tab[mid].z, tab[mid].yx) < lo) l = mid + 1;
        else h = mid;
    }
    for (int k = l; k < e; ++k) {
        const PtEntry en = tab[k];
        if (entry_key(en.z, en.yx) >= hi) break;
        f(en.yx & 3, en);
    }
}

// Laplacian sum of 4 consecutive columns col0 .. col0+3 of shared-memory row zl
// (row width SW floats, at least round4(M) columns of halo on either side of
// them, col0 a multiple of 4); cc receives the centre values.
template <int SHAPE, int M, int NN, int SW, class PP>
__device__ __forceinline__ void lap2d_at(const PP &p, const float *sm, int zl, int col0,
                                         float (&cc)[4], float (&lap)[4])
{
    constexpr int HX = round4(M);
    const float4 c = ld4(sm + zl * SW + col0);
    cc[0] = c.x; cc[1] = c.y; cc[2] = c.z; cc[3] = c.w;
    float u2[4], u4[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        u2[j] = cc[j] + cc[j];
        u4[j] = u2[j] + u2[j];
    }
    // Centre-free Laplacian: sum_o a_o (u(x+o) - u(x)), the same sum since
    // the weights of a consistent stencil add up to zero.  Each group of n
    // points has n u(x) subtracted before it is weighted, so a constant
    // field gives exactly zero whatever the FP32 rounding of the weights,
    // and the accumulator only holds small differences.
    lap[0] = lap[1] = lap[2] = lap[3] = 0.f;
    if (SHAPE == FD_CROSS) {
        // x and z arms of offset m share the weight W[0][m]
        float win[4 + 2 * HX];
#pragma unroll
        for (int i = 0; i < (4 + 2 * HX) / 4; ++i) {
            const float4 a = ld4(sm + zl * SW + col0 - HX + 4 * i);
            win[4 * i] = a.x; win[4 * i + 1] = a.y; win[4 * i + 2] = a.z; win[4 * i + 3] = a.w;
        }
#pragma unroll
        for (int m = 1; m <= M; ++m) {
            const float4 a = ld4(sm + (zl + m) * SW + col0);
            const float4 b = ld4(sm + (zl - m) * SW + col0);
            const float zp[4] = {a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w};
#pragma unroll
            for (int j = 0; j < 4; ++j)
                lap[j] = fmaf(p.w[m], ((win[HX + j + m] + win[HX + j - m]) + zp[j]) - u4[j],
                              lap[j]);
        }
    } else {
#pragma unroll
        for (int q = 0; q <= M; ++q) {
            const int E = shape_ext(SHAPE, M, NN, q);
            if (E < 0) continue;
            const int E4 = round4(E);
            float win[4 + 2 * round4(M)];
            const float *rp = sm + (zl + q) * SW + col0 - E4;
            const float *rm = sm + (zl - q) * SW + col0 - E4;
#pragma unroll
            for (int i = 0; i < (4 + 2 * E4) / 4; ++i) {
                float4 a = ld4(rp + 4 * i);
                if (q > 0) {
                    const float4 b = ld4(rm + 4 * i);
                    a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
                }
                win[4 * i] = a.x; win[4 * i + 1] = a.y; win[4 * i + 2] = a.z; win[4 * i + 3] = a.w;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                // row pair z +- q holds 2 points at dx = 0 and 4 at dx = +-pp;
                // row z holds the centre (no term) and 2 points at +-pp
                const float un = q > 0 ? u4[j] : u2[j];
                float acc = q > 0 ? p.w[q] * (win[E4 + j] - u2[j]) : 0.f;   // W[0][q]
#pragma unroll
                for (int pp = 1; pp <= E; ++pp)
                    acc = fmaf(p.w[pp * kWDim + q], (win[E4 + j + pp] + win[E4 + j - pp]) - un, acc);
                lap[j] += acc;
            }
        }
    }
}

// The same for thread column tx of a tile staged with its halo (row width
// kTX + 2 round4(M)).
template <int SHAPE, int M, int NN, class PP>
__device__ __forceinline__ void lap2d_row(const PP &p, const float *sm, int zl, int tx,
                                          float (&cc)[4], float (&lap)[4])
{
    lap2d_at<SHAPE, M, NN, kTX + 2 * round4(M)>(p, sm, zl, round4(M) + 4 * tx, cc, lap);
}

// One tile of the 2D step.  PP is the parameter view: StepParams for a
// single-shot launch, BatchView (below) for a launch over many shots.
template <int SHAPE, int M, int NN, int MODE, int R, class PP>
__device__ __forceinline__ void step2d_tile(const PP &p, const int tile, float *sm, uint64_t &bar)
{
    constexpr int HX = round4(M);
    constexpr int SW = kTX + 2 * HX;
    constexpr int SH = kTZ * R + 2 * M;

    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int x0 = (tile % p.tiles_x) * kTX;
    const int z0 = (tile / p.tiles_x) * (kTZ * R);

    if (threadIdx.x == 0) {
        prefetch_tmap(p.tmap);
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, SW * SH * 4);
        tma_load_2d(sm, p.tmap, &bar, x0 - HX, z0 - M);
    }

    const int xg = x0 + 4 * tx;
    const bool colok = xg < p.nx;
    float4 up[R], kp[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int zg = z0 + ty * R + r;
        if (colok && zg < p.nz) {
            const int64_t o = (int64_t)zg * p.pitch + xg;
            up[r] = ldg4(p.u_prev + o);
            kp[r] = ldg4(p.kappa + o);
        } else {
            up[r] = make_float4(0.f, 0.f, 0.f, 0.f);
            kp[r] = up[r];
        }
    }
    float d2x[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) d2x[j] = layer_d2(xg + j, p.phys_lo[0], p.phys_hi[0]);
    // the tile's ranges in the point tables, read once while the copy is in
    // flight; most tiles have empty ranges and touch the tables no further
    const int ib = p.inj_ptr ? p.inj_ptr[tile] : 0, ie = p.inj_ptr ? p.inj_ptr[tile + 1] : 0;
    const int sb = p.smp_ptr ? p.smp_ptr[tile] : 0, se = p.smp_ptr ? p.smp_ptr[tile + 1] : 0;

    const bool ok = mbar_wait_bounded(&bar, 0);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
            atomicOr(p.status, kStatusTimeout);
            mbar_wait_bounded(&bar, 0);   // let an in-flight copy land before exiting
        }
        return;
    }

#pragma unroll 1
    for (int r = 0; r < R; ++r) {
        const int zl = M + ty * R + r;
        const int zg = z0 + ty * R + r;
        float cc[4], lap[4];
        lap2d_row<SHAPE, M, NN>(p, sm, zl, tx, cc, lap);
        const float d2z = layer_d2(zg, p.phys_lo[2], p.phys_hi[2]);
        const float uu[4] = {up[r].x, up[r].y, up[r].z, up[r].w};
        const float kk[4] = {kp[r].x, kp[r].y, kp[r].z, kp[r].w};
        float o[4], dv[4], g[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            g[j] = sponge_g(p.gcoef, d2x[j] + d2z);
            dv[j] = step_update(cc[j], uu[j], kk[j], lap[j], g[j], o[j]);
        }
        // injection inside the bracket; adjoint residuals are scaled by kappa
        if (ib < ie)
            for_row(p.inj, ib, ie, zg, tx, [&](int j, const PtEntry &en) {
                float a = src_term(en.scale, p.inj_series[(int64_t)p.step * p.inj_ncol + en.col]);
                if (MODE == kModeAdjoint) a = __fmul_rn(a, kk[j]);
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
                    if (jj == j) o[jj] = __fadd_rn(o[jj], a);
            });
#pragma unroll
        for (int j = 0; j < 4; ++j)
            o[j] = sponge_div(o[j], g[j]);
        if (sb < se)
            for_row(p.smp, sb, se, zg, tx, [&](int j, const PtEntry &en) {
                float v = 0.f;
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
                    if (jj == j) v = o[jj];
                v *= en.scale;
                if (MODE == kModeAdjoint) v /= kk[j];
                p.smp_out[(int64_t)p.step * p.smp_ncol + en.col] = v;
            });
        if (!colok || zg >= p.nz) continue;
        const int64_t off = (int64_t)zg * p.pitch + xg;
        const float4 un = make_float4(o[0], o[1], o[2], o[3]);
        if (p.check) check_growth(p.status, un);
        *reinterpret_cast<float4 *>(p.u_prev + off) = un;
        if (MODE != kModeAdjoint && p.dseg_out)
            *reinterpret_cast<float4 *>(p.dseg_out + off) = make_float4(dv[0], dv[1], dv[2], dv[3]);
        if (MODE == kModeAdjoint) {
            const float4 d = ldg4(p.dseg_in + off);
            float4 ga = *reinterpret_cast<float4 *>(p.gacc + off);
            ga.x = fmaf(un.x, d.x, ga.x); ga.y = fmaf(un.y, d.y, ga.y);
            ga.z = fmaf(un.z, d.z, ga.z); ga.w = fmaf(un.w, d.w, ga.w);
            *reinterpret_cast<float4 *>(p.gacc + off) = ga;
        }
    }
}

template <int SHAPE, int M, int NN, int MODE, int R>
__global__ void __launch_bounds__(kThreads) step2d_kernel(const __grid_constant__ StepParams p)
{
    extern __shared__ __align__(1024) float sm[];
    __shared__ uint64_t bar;
    step2d_tile<SHAPE, M, NN, MODE, R>(p, blockIdx.x, sm, bar);
}

// ---------------------------------------------------------------------------
// Batched shots: one launch per time step over the tiles of every shot.  The
// CTAs are persistent and walk the tile table with a stride of gridDim.x.  A
// producer warp stages each tile in one of NB shared-memory slots: by TMA the
// halo box of u^n and the u^{n-1} and kappa tiles, and by plain copies the
// shot's scalars and the tile's ranges in the point tables; each slot has a
// full and an empty mbarrier, so the copies of the next tiles overlap the
// arithmetic of the current one.  The weights stay in kernel parameters.
// ---------------------------------------------------------------------------
struct BatchView {
    float *u_prev;
    float *dseg;               // D of this step (store-D and adjoint modes)
    float *gacc;
    int64_t nx, nz, pitch;
    int64_t phys_lo[3], phys_hi[3];
    float gcoef;
    int tiles_x;
    const PtEntry *inj;
    const float *inj_series;
    int inj_ncol;
    const PtEntry *smp;
    float *smp_out;
    int smp_ncol;
    int step;
    int check;
    int *status;
    const float (&w)[kWDim * kWDim];
    __device__ BatchView(const ShotInfo &d, const BatchParams &bp)
        : BatchView(d, bp, bp.step, bp.parity, bp.check) {}
    // the same with the step, field parity and growth check given explicitly
    // (the persistent batched kernel advances them itself)
    __device__ BatchView(const ShotInfo &d, const BatchParams &bp, int step_, int parity, int check_)
        : u_prev(d.buf[parity ^ 1]), dseg(d.dseg ? d.dseg + (int64_t)bp.seg * d.field : nullptr),
          gacc(d.gacc), nx(d.nx), nz(d.nz), pitch(d.pitch), gcoef(d.gcoef),
          tiles_x(d.tiles_x), inj(d.inj), inj_series(d.inj_series), inj_ncol(d.inj_ncol),
          smp(d.smp), smp_out(d.smp_out), smp_ncol(d.smp_ncol), step(step_), check(check_),
          status(bp.status), w(bp.w)
    {
        for (int i = 0; i < 3; ++i) {
            phys_lo[i] = d.phys_lo[i];
            phys_hi[i] = d.phys_hi[i];
        }
    }
};

// What the producer warp stages for a slot besides the field data: the
// shot's scalars, the tile and its ranges in the injection and sampling tables.
struct Staged {
    ShotInfo info;
    TileRec rec;
};

template <int M, int R>
struct StreamCfg {
    static constexpr int HX = round4(M);
    static constexpr int SW = kTX + 2 * HX;
    static constexpr int SH = kTZ * R + 2 * M;
    static constexpr int AEL = (SW * SH + 31) & ~31;   // halo box, 128-byte padded
    static constexpr int TEL = kTX * kTZ * R;          // one tile
    static constexpr int SLOT = AEL + 2 * TEL;         // halo box | u_prev tile | kappa tile
    // as many slots (2 to 4) as fit in about 74 KB, so that three CTAs share
    // an SM (their registers allow three) and each keeps up to NB - 1 tiles of
    // copies in flight
    static constexpr int NB = 74 * 1024 / (SLOT * 4) < 2 ? 2
                            : 74 * 1024 / (SLOT * 4) > 4 ? 4 : 74 * 1024 / (SLOT * 4);
    static constexpr size_t SMEM = (size_t)NB * SLOT * sizeof(float);
    static constexpr int NCW = kThreads / 32;          // consumer warps
    static constexpr int THREADS = kThreads + 32;
};

// One step of one staged tile: forward (MODE kModeForward), forward storing
// D = kappa lap (kModeStoreD) or adjoint with the gradient accumulation
// (kModeAdjoint), with the arithmetic of step2d_tile in each mode.  CHECK
// false compiles the growth check out (the per-step batched kernel runs the
// checking instantiation on the checking steps only).
template <int SHAPE, int M, int R, int MODE, bool CHECK = true>
__device__ __forceinline__ void stream_tile(const BatchView &v, const Staged &st,
                                            const float *slot, int tx, int ty)
{
    using C = StreamCfg<M, R>;
    const int x0 = st.rec.x0, z0 = st.rec.z0;
    const int xg = x0 + 4 * tx;
    const bool colok = xg < v.nx;
    float d2x[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) d2x[j] = layer_d2(xg + j, v.phys_lo[0], v.phys_hi[0]);
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
        const int rr = ty * R + r;
        const int zg = z0 + rr;
        float cc[4], lap[4];
        lap2d_row<SHAPE, M, 0>(v, slot, M + rr, tx, cc, lap);
        const float4 up = ld4(slot + C::AEL + rr * kTX + 4 * tx);
        const float4 kp = ld4(slot + C::AEL + C::TEL + rr * kTX + 4 * tx);
        const float uu[4] = {up.x, up.y, up.z, up.w};
        const float kk[4] = {kp.x, kp.y, kp.z, kp.w};
        const float d2z = layer_d2(zg, v.phys_lo[2], v.phys_hi[2]);
        float o[4], dv[4], g[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            g[j] = sponge_g(v.gcoef, d2x[j] + d2z);
            dv[j] = step_update(cc[j], uu[j], kk[j], lap[j], g[j], o[j]);
        }
        if (st.rec.ib < st.rec.ie)
            for_row(v.inj, st.rec.ib, st.rec.ie, zg, tx, [&](int j, const PtEntry &en) {
                float a = src_term(en.scale, v.inj_series[(int64_t)v.step * v.inj_ncol + en.col]);
                if (MODE == kModeAdjoint) a = __fmul_rn(a, kk[j]);
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
                    if (jj == j) o[jj] = __fadd_rn(o[jj], a);
            });
#pragma unroll
        for (int j = 0; j < 4; ++j)
            o[j] = sponge_div(o[j], g[j]);
        if (st.rec.sb < st.rec.se)
            for_row(v.smp, st.rec.sb, st.rec.se, zg, tx, [&](int j, const PtEntry &en) {
                float s = 0.f;
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
                    if (jj == j) s = o[jj];
                s *= en.scale;
                if (MODE == kModeAdjoint) s /= kk[j];
                v.smp_out[(int64_t)v.step * v.smp_ncol + en.col] = s;
            });
        if (!colok || zg >= v.nz) continue;
        const int64_t off = (int64_t)zg * v.pitch + xg;
        const float4 un = make_float4(o[0], o[1], o[2], o[3]);
        if (CHECK && v.check) check_growth(v.status, un);
        *reinterpret_cast<float4 *>(v.u_prev + off) = un;
        if (MODE == kModeStoreD)
            *reinterpret_cast<float4 *>(v.dseg + off) = make_float4(dv[0], dv[1], dv[2], dv[3]);
        if (MODE == kModeAdjoint) {
            const float4 d = ldg4(v.dseg + off);
            float4 ga = *reinterpret_cast<float4 *>(v.gacc + off);
            ga.x = fmaf(un.x, d.x, ga.x); ga.y = fmaf(un.y, d.y, ga.y);
            ga.z = fmaf(un.z, d.z, ga.z); ga.w = fmaf(un.w, d.w, ga.w);
            *reinterpret_cast<float4 *>(v.gacc + off) = ga;
        }
    }
}

template <int SHAPE, int M, int R, int MODE, bool CHECK>
__global__ void __launch_bounds__(StreamCfg<M, R>::THREADS)
step2d_batched(const __grid_constant__ BatchParams bp)
{
    using C = StreamCfg<M, R>;
    constexpr int NB = C::NB;
    constexpr uint32_t BYTES = (C::SW * C::SH + 2 * C::TEL) * 4;
    extern __shared__ __align__(1024) float sm[];
    __shared__ uint64_t full[NB], empty[NB];
    __shared__ Staged staged[NB];
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int i = 0; i < NB; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], C::NCW);
        }
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    const int G = gridDim.x;
    const int cur = bp.parity;

    if (warp == C::NCW) {   // producer: lane 0 waits and issues, the warp copies
        volatile int *abort_v = &abort_flag;
        constexpr int kWords = sizeof(ShotInfo) / 4;
        int i = 0;
        TileRec next = blockIdx.x < bp.ntiles ? bp.tiles[blockIdx.x] : TileRec{};
        for (int g = blockIdx.x; g < bp.ntiles; g += G, ++i) {
            const int b = i % NB;
            const TileRec rec = next;
            if (g + G < bp.ntiles) next = bp.tiles[g + G];     // one record ahead
            int go = 1;
            if (lane == 0) {
                if (i >= NB && !mbar_wait_bounded(&empty[b], (uint32_t)((i / NB - 1) & 1))) {
                    atomicOr(bp.status, kStatusTimeout);
                    *abort_v = 1;
                }
                go = !*abort_v;
            }
            if (!__shfl_sync(0xffffffffu, go, 0)) break;
            const ShotDesc &d = bp.shots[rec.shot];
            if (lane == 0) {   // field data first; the arrival below closes the phase
                float *fd = sm + b * C::SLOT;
                mbar_expect_tx(&full[b], BYTES);
                tma_load_2d(fd, &d.tmap[cur], &full[b], rec.x0 - C::HX, rec.z0 - M);
                tma_load_2d(fd + C::AEL, &d.tile[cur ^ 1], &full[b], rec.x0, rec.z0);
                tma_load_2d(fd + C::AEL + C::TEL, &d.ktile, &full[b], rec.x0, rec.z0);
                staged[b].rec = rec;
            }
            const uint32_t *src = reinterpret_cast<const uint32_t *>(&d.info);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&staged[b].info);
            for (int k = lane; k < kWords; k += 32) dst[k] = src[k];
            __syncwarp();
            if (lane == 0) {
                // the staged words above are released to the consumers by the arrive
                __threadfence_block();
                mbar_arrive(&full[b]);
            }
        }
        if (lane == 0 && *abort_v) {   // let the copies in flight land before the block exits
            for (int j = i > NB ? i - NB : 0; j < i; ++j)
                mbar_wait_bounded(&full[j % NB], (j / NB) & 1, 100000000LL);
        }
        return;
    }

    const int tx = tid & 15, ty = tid >> 4;
    bool ok = true;
    int i = 0;
    for (int g = blockIdx.x; g < bp.ntiles; g += G, ++i) {
        const int b = i % NB;
        if (*reinterpret_cast<volatile int *>(&abort_flag)) break;
        ok = mbar_wait_bounded(&full[b], (i / NB) & 1);
        if (!ok) break;
        const BatchView v(staged[b].info, bp);
        stream_tile<SHAPE, M, R, MODE, CHECK>(v, staged[b], sm + b * C::SLOT, tx, ty);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[b]);
    }
    if (!ok) {
        atomicOr(bp.status, kStatusTimeout);
        *reinterpret_cast<volatile int *>(&abort_flag) = 1;
    }
}

// ---------------------------------------------------------------------------
// Batched shots, every time step in one persistent launch.  A cooperative
// launch keeps all CTAs resident; each walks its share of the tile table for
// step n through the same producer/consumer ring as step2d_batched (the ring
// position carries over from step to step), then the CTAs meet at a grid
// barrier before step n + 1 reads what step n wrote.  The barrier's words are
// the status block's words 1 (abort), 2 (count) and 3 (generation).  Every
// wait is bounded: a time-out sets the status bit and the abort word, the
// producer lets its copies in flight land, and every CTA leaves at its next
// barrier.  The TMA-issuing lane orders the previous step's generic-proxy
// writes before its async-proxy reads with a proxy fence after the barrier.
// Same per-point arithmetic as the per-step kernel, so the same bits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool batch_grid_sync(const BatchParams &bp, bool local_abort)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = local_abort ? 0 : 1;
        volatile int *abort_g = bp.status + 1;
        unsigned int *count = reinterpret_cast<unsigned int *>(bp.status + 2);
        volatile unsigned int *gen = reinterpret_cast<volatile unsigned int *>(bp.status + 3);
        if (!ok) {
            *abort_g = 1;
        } else {
            const unsigned int g = *gen;
            __threadfence();
            const unsigned int a = atomicAdd(count, 1u) + 1u;
            if (a == gridDim.x) {
                atomicExch(count, 0u);
                __threadfence();
                atomicAdd(reinterpret_cast<unsigned int *>(bp.status + 3), 1u);
            } else {
                const long long t0 = clock64();
                while (*gen == g) {
                    if (*abort_g) {
                        ok = 0;
                        break;
                    }
                    if (clock64() - t0 > kWaitCycles) {
                        atomicOr(bp.status, kStatusTimeout);
                        *abort_g = 1;
                        ok = 0;
                        break;
                    }
                    __nanosleep(32);
                }
            }
            __threadfence();
        }
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

template <int SHAPE, int M, int R>
__global__ void __launch_bounds__(StreamCfg<M, R>::THREADS)
step2d_batched_persistent(const __grid_constant__ BatchParams bp, int nt)
{
    using C = StreamCfg<M, R>;
    constexpr int NB = C::NB;
    constexpr uint32_t BYTES = (C::SW * C::SH + 2 * C::TEL) * 4;
    extern __shared__ __align__(1024) float sm[];
    __shared__ uint64_t full[NB], empty[NB];
    __shared__ Staged staged[NB];
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int i = 0; i < NB; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], C::NCW);
        }
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    const int G = gridDim.x;
    volatile int *abort_v = &abort_flag;
    const int tx = tid & 15, ty = tid >> 4;
    int i = 0;   // ring position; producer and consumers count the same tiles
    for (int n = 0; n < nt; ++n) {
        const int cur = n & 1;
        const int check = (n + 1) % kCheckEvery == 0 || n + 1 == nt;
        if (warp == C::NCW) {   // producer: lane 0 waits and issues, the warp copies
            constexpr int kWords = sizeof(ShotInfo) / 4;
            if (lane == 0) asm volatile("fence.proxy.async.global;" ::: "memory");
            TileRec next = blockIdx.x < bp.ntiles ? bp.tiles[blockIdx.x] : TileRec{};
            for (int g = blockIdx.x; g < bp.ntiles; g += G, ++i) {
                const int b = i % NB;
                const TileRec rec = next;
                if (g + G < bp.ntiles) next = bp.tiles[g + G];
                int go = 1;
                if (lane == 0) {
                    if (i >= NB && !mbar_wait_bounded(&empty[b], (uint32_t)((i / NB - 1) & 1))) {
                        atomicOr(bp.status, kStatusTimeout);
                        *abort_v = 1;
                    }
                    go = !*abort_v;
                }
                if (!__shfl_sync(0xffffffffu, go, 0)) break;
                const ShotDesc &d = bp.shots[rec.shot];
                if (lane == 0) {
                    float *fd = sm + b * C::SLOT;
                    mbar_expect_tx(&full[b], BYTES);
                    tma_load_2d(fd, &d.tmap[cur], &full[b], rec.x0 - C::HX, rec.z0 - M);
                    tma_load_2d(fd + C::AEL, &d.tile[cur ^ 1], &full[b], rec.x0, rec.z0);
                    tma_load_2d(fd + C::AEL + C::TEL, &d.ktile, &full[b], rec.x0, rec.z0);
                    staged[b].rec = rec;
                }
                const uint32_t *src = reinterpret_cast<const uint32_t *>(&d.info);
                uint32_t *dst = reinterpret_cast<uint32_t *>(&staged[b].info);
                for (int k = lane; k < kWords; k += 32) dst[k] = src[k];
                __syncwarp();
                if (lane == 0) {
                    __threadfence_block();
                    mbar_arrive(&full[b]);
                }
            }
            if (lane == 0 && *abort_v) {   // let the copies in flight land before leaving
                for (int j = i > NB ? i - NB : 0; j < i; ++j)
                    mbar_wait_bounded(&full[j % NB], (j / NB) & 1, 100000000LL);
            }
        } else {
            bool ok = true;
            for (int g = blockIdx.x; g < bp.ntiles; g += G, ++i) {
                const int b = i % NB;
                if (*abort_v) break;
                ok = mbar_wait_bounded(&full[b], (i / NB) & 1);
                if (!ok) break;
                const BatchView v(staged[b].info, bp, n, cur, check);
                stream_tile<SHAPE, M, R, kModeForward>(v, staged[b], sm + b * C::SLOT, tx, ty);
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[b]);
            }
            if (!ok) {
                atomicOr(bp.status, kStatusTimeout);
                *abort_v = 1;
            }
        }
        if (!batch_grid_sync(bp, *abort_v != 0)) return;
    }
}

// ---------------------------------------------------------------------------
// Batched shots, two time steps per pass (temporal blocking).  Each tile is
// staged with the halo that two steps need: u^n with 2M rows (and
// round4(HX + M) columns) around it, u^{n-1} and kappa with M rows (and HX
// columns).  The consumers first compute u^{n+1} on the tile plus its M-row
// halo ("extended region", kept in shared memory; halo points are computed
// redundantly by every tile that needs them, with the same arithmetic as
// their owner), then u^{n+2} on the tile from it.  Both results are written
// to two buffers other than the inputs (four buffers in rotation), so no
// tile overwrites data another tile still reads.  Per step this moves 10
// bytes per point through HBM instead of 16.  Outside the grid the staged
// fields and kappa are zero, so u^{n+1} there is exactly zero, as the
// boundary condition requires.
// ---------------------------------------------------------------------------
template <int M, int R>
struct Stream2Cfg {
    static constexpr int TZ = kTZ * R;
    static constexpr int HX = round4(M);
    static constexpr int HXC = round4(HX + M);
    static constexpr int EW = kTX + 2 * HX, EH = TZ + 2 * M;      // extended region
    static constexpr int CW = kTX + 2 * HXC, CH = TZ + 4 * M;     // u^n box
    static constexpr int CEL = (CW * CH + 31) & ~31;
    static constexpr int EEL = (EW * EH + 31) & ~31;
    static constexpr int SLOT = CEL + 2 * EEL;                    // u^n | u^{n-1} | kappa
    static constexpr int NB = 2;
    static constexpr int NCW = kThreads / 32;
    static constexpr int THREADS = kThreads + 32;
    static constexpr size_t SMEM = ((size_t)NB * SLOT + EEL) * sizeof(float);
};

// Barrier of the consumer warps only (named barrier 1; the producer warp does
// not take part), and the same with an OR over a predicate.
__device__ __forceinline__ void consumers_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory");
}

__device__ __forceinline__ bool consumers_any(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kThreads)
        : "memory");
    return r != 0;
}

template <int SHAPE, int M, int R>
__device__ __forceinline__ void stream2_tile(const BatchView &v, const Staged &st,
                                             const PtEntry *ext, const float *slot, float *u1,
                                             float *out1, float *out2, int tid)
{
    using C = Stream2Cfg<M, R>;
    const int x0 = st.rec.x0, z0 = st.rec.z0;
    const int ex0 = x0 - C::HX, ez0 = z0 - M;            // extended region origin
    const float *cur = slot, *prv = slot + C::CEL, *kap = slot + C::CEL + C::EEL;
    // stage 1: u^{n+1} on the extended region (groups of 4 columns)
    constexpr int GX = C::EW / 4, ITEMS = GX * C::EH;
#pragma unroll 1
    for (int it = tid; it < ITEMS; it += kThreads) {
        const int gx = it % GX, rz = it / GX;
        const int c0 = 4 * gx;
        const int zg = ez0 + rz;
        float cc[4], lap[4];
        lap2d_at<SHAPE, M, 0, C::CW>(v, cur, rz + M, c0 + (C::HXC - C::HX), cc, lap);
        const float4 up = ld4(prv + rz * C::EW + c0);
        const float4 kp = ld4(kap + rz * C::EW + c0);
        const float uu[4] = {up.x, up.y, up.z, up.w};
        const float kk[4] = {kp.x, kp.y, kp.z, kp.w};
        const float d2z = layer_d2(zg, v.phys_lo[2], v.phys_hi[2]);
        float o[4], g[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            g[j] = sponge_g(v.gcoef, layer_d2(ex0 + c0 + j, v.phys_lo[0], v.phys_hi[0]) + d2z);
            step_update(cc[j], uu[j], kk[j], lap[j], g[j], o[j]);
        }
        for (int k = st.rec.xb; k < st.rec.xe; ++k) {
            const PtEntry en = ext[k];
            const int xl = en.yx & 0xffff;
            if (en.z != zg || (xl >> 2) != gx) continue;
            const float a = src_term(en.scale, v.inj_series[(int64_t)v.step * v.inj_ncol + en.col]);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
                if (jj == (xl & 3)) o[jj] = __fadd_rn(o[jj], a);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            o[j] = sponge_div(o[j], g[j]);
        *reinterpret_cast<float4 *>(u1 + rz * C::EW + c0) = make_float4(o[0], o[1], o[2], o[3]);
        // points of the tile itself: store and sample step n
        const int tr = rz - M, tc = c0 - C::HX;
        if (tr < 0 || tr >= C::TZ || tc < 0 || tc >= kTX) continue;
        if (st.rec.sb < st.rec.se)
            for_row(v.smp, st.rec.sb, st.rec.se, zg, tc >> 2, [&](int j, const PtEntry &en) {
                float sv = 0.f;
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
                    if (jj == j) sv = o[jj];
                v.smp_out[(int64_t)v.step * v.smp_ncol + en.col] = sv * en.scale;
            });
        const int xg = x0 + tc;
        if (xg < v.nx && zg < v.nz) {
            const float4 un = make_float4(o[0], o[1], o[2], o[3]);
            if (v.check) check_growth(v.status, un);
            *reinterpret_cast<float4 *>(out1 + (int64_t)zg * v.pitch + xg) = un;
        }
    }
    consumers_sync();
    // stage 2: u^{n+2} on the tile
    const int tx = tid & 15, ty = tid >> 4;
    const int xg = x0 + 4 * tx;
    const bool colok = xg < v.nx;
    const int step1 = v.step + 1;
    float d2x[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) d2x[j] = layer_d2(xg + j, v.phys_lo[0], v.phys_hi[0]);
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
        const int rr = ty * R + r;
        const int zg = z0 + rr;
        float cc[4], lap[4];
        lap2d_at<SHAPE, M, 0, C::EW>(v, u1, rr + M, C::HX + 4 * tx, cc, lap);
        const float4 up = ld4(cur + (rr + 2 * M) * C::CW + C::HXC + 4 * tx);
        const float4 kp = ld4(kap + (rr + M) * C::EW + C::HX + 4 * tx);
        const float uu[4] = {up.x, up.y, up.z, up.w};
        const float kk[4] = {kp.x, kp.y, kp.z, kp.w};
        const float d2z = layer_d2(zg, v.phys_lo[2], v.phys_hi[2]);
        float o[4], g[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            g[j] = sponge_g(v.gcoef, d2x[j] + d2z);
            step_update(cc[j], uu[j], kk[j], lap[j], g[j], o[j]);
        }
        for (int k = st.rec.xb; k < st.rec.xe; ++k) {
            const PtEntry en = ext[k];
            const int xl = (en.yx & 0xffff) - C::HX;
            if (en.z != zg || xl < 0 || (xl >> 2) != tx) continue;
            const float a = src_term(en.scale, v.inj_series[(int64_t)step1 * v.inj_ncol + en.col]);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
                if (jj == (xl & 3)) o[jj] = __fadd_rn(o[jj], a);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            o[j] = sponge_div(o[j], g[j]);
        if (st.rec.sb < st.rec.se)
            for_row(v.smp, st.rec.sb, st.rec.se, zg, tx, [&](int j, const PtEntry &en) {
                float sv = 0.f;
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
                    if (jj == j) sv = o[jj];
                v.smp_out[(int64_t)step1 * v.smp_ncol + en.col] = sv * en.scale;
            });
        if (!colok || zg >= v.nz) continue;
        const float4 un = make_float4(o[0], o[1], o[2], o[3]);
        if (v.check) check_growth(v.status, un);
        *reinterpret_cast<float4 *>(out2 + (int64_t)zg * v.pitch + xg) = un;
    }
    consumers_sync();   // u1 is rewritten by the next tile
}

template <int SHAPE, int M, int R>
__global__ void __launch_bounds__(Stream2Cfg<M, R>::THREADS)
step2d_batched2(const __grid_constant__ BatchParams bp)
{
    using C = Stream2Cfg<M, R>;
    constexpr int NB = C::NB;
    constexpr uint32_t BYTES = (C::CW * C::CH + 2 * C::EW * C::EH) * 4;
    extern __shared__ __align__(1024) float sm[];
    __shared__ uint64_t full[NB], empty[NB];
    __shared__ Staged staged[NB];
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int i = 0; i < NB; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], C::NCW);
        }
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    const int G = gridDim.x;
    const int rc = bp.roles[0], rp = bp.roles[1];

    if (warp == C::NCW) {   // producer: lane 0 waits and issues, the warp copies
        volatile int *abort_v = &abort_flag;
        constexpr int kWords = sizeof(ShotInfo) / 4;
        int i = 0;
        TileRec next = blockIdx.x < bp.ntiles ? bp.tiles[blockIdx.x] : TileRec{};
        for (int g = blockIdx.x; g < bp.ntiles; g += G, ++i) {
            const int b = i % NB;
            const TileRec rec = next;
            if (g + G < bp.ntiles) next = bp.tiles[g + G];
            int go = 1;
            if (lane == 0) {
                if (i >= NB && !mbar_wait_bounded(&empty[b], (uint32_t)((i / NB - 1) & 1))) {
                    atomicOr(bp.status, kStatusTimeout);
                    *abort_v = 1;
                }
                go = !*abort_v;
            }
            if (!__shfl_sync(0xffffffffu, go, 0)) break;
            const ShotDesc &d = bp.shots[rec.shot];
            if (lane == 0) {
                float *fd = sm + b * C::SLOT;
                mbar_expect_tx(&full[b], BYTES);
                tma_load_2d(fd, &d.c2[rc], &full[b], rec.x0 - C::HXC, rec.z0 - 2 * M);
                tma_load_2d(fd + C::CEL, &d.p2[rp], &full[b], rec.x0 - C::HX, rec.z0 - M);
                tma_load_2d(fd + C::CEL + C::EEL, &d.k2, &full[b], rec.x0 - C::HX, rec.z0 - M);
                staged[b].rec = rec;
            }
            const uint32_t *src = reinterpret_cast<const uint32_t *>(&d.info);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&staged[b].info);
            for (int k = lane; k < kWords; k += 32) dst[k] = src[k];
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                mbar_arrive(&full[b]);
            }
        }
        if (lane == 0 && *abort_v) {
            for (int j = i > NB ? i - NB : 0; j < i; ++j)
                mbar_wait_bounded(&full[j % NB], (j / NB) & 1, 100000000LL);
        }
        return;
    }

    float *u1 = sm + NB * C::SLOT;
    bool ok = true;
    int i = 0;
    for (int g = blockIdx.x; g < bp.ntiles; g += G, ++i) {
        const int b = i % NB;
        ok = mbar_wait_bounded(&full[b], (i / NB) & 1);
        // every consumer warp takes part in the named barriers of a tile, so
        // they decide together whether to go on (each wait above is bounded)
        if (consumers_any(!ok || *reinterpret_cast<volatile int *>(&abort_flag))) {
            ok = false;
            break;
        }
        const Staged &st = staged[b];
        const BatchView v(st.info, bp);
        stream2_tile<SHAPE, M, R>(v, st, bp.ext, sm + b * C::SLOT, u1, st.info.buf[bp.roles[2]],
                                  st.info.buf[bp.roles[3]], tid);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[b]);
    }
    if (!ok) {
        atomicOr(bp.status, kStatusTimeout);
        *reinterpret_cast<volatile int *>(&abort_flag) = 1;
    }
}

// ---------------------------------------------------------------------------
// Persistent time loop for small grids (fields resident in L2), where the
// latency of one launch per step dominates: a cooperative launch keeps every
// CTA resident; CTAs loop over the time steps and take their tiles of each
// step in turn, separated by a grid barrier.  The barrier spins with a time
// bound and an abort flag: on a time-out the status bit is set, the flag
// raised, and every CTA leaves at its next barrier.  After the barrier the
// TMA-issuing thread executes a generic->async proxy fence, so the field
// written in the previous step by other CTAs is what the next TMA loads read.
// ---------------------------------------------------------------------------
struct StepView {
    const CUtensorMap *tmap;
    float *u_prev;
    const float *kappa;
    int64_t nx, nz, pitch;
    int64_t phys_lo[3], phys_hi[3];
    float gcoef;
    int tiles_x;
    const int32_t *inj_ptr;
    const PtEntry *inj;
    const float *inj_series;
    int inj_ncol;
    const int32_t *smp_ptr;
    const PtEntry *smp;
    float *smp_out;
    int smp_ncol;
    int step;
    int check;
    float *dseg_out;
    const float *dseg_in;
    float *gacc;
    int *status;
    const float (&w)[kWDim * kWDim];
    __device__ StepView(const PersistParams &pp, int n)
        : tmap(pp.maps + 2 * (n & 1)), u_prev(pp.buf[(n & 1) ^ 1]), kappa(pp.base.kappa),
          nx(pp.base.nx), nz(pp.base.nz), pitch(pp.base.pitch), gcoef(pp.base.gcoef),
          tiles_x(pp.base.tiles_x), inj_ptr(pp.base.inj_ptr), inj(pp.base.inj),
          inj_series(pp.base.inj_series), inj_ncol(pp.base.inj_ncol), smp_ptr(pp.base.smp_ptr),
          smp(pp.base.smp), smp_out(pp.base.smp_out), smp_ncol(pp.base.smp_ncol), step(n),
          check((n + 1) % kCheckEvery == 0 || n + 1 == pp.nt), dseg_out(nullptr), dseg_in(nullptr), gacc(nullptr), status(pp.base.status), w(pp.base.w)
    {
        for (int i = 0; i < 3; ++i) {
            phys_lo[i] = pp.base.phys_lo[i];
            phys_hi[i] = pp.base.phys_hi[i];
        }
    }
};

// Grid-wide barrier; false if it timed out here or another CTA aborted.
__device__ __forceinline__ bool grid_sync(const PersistParams &pp)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned int *gen = pp.bar_gen;
        volatile int *abort_v = pp.abort_flag;
        const unsigned int g = *gen;
        __threadfence();
        const unsigned int a = atomicAdd(pp.bar_count, 1u) + 1u;
        if (a == gridDim.x) {
            atomicExch(pp.bar_count, 0u);
            __threadfence();
            atomicAdd(pp.bar_gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g) {
                if (*abort_v) {
                    ok = 0;
                    break;
                }
                if (clock64() - t0 > 4000000000LL) {
                    atomicOr(pp.base.status, kStatusTimeout);
                    *abort_v = 1;
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        asm volatile("fence.proxy.async.global;" ::: "memory");
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

template <int SHAPE, int M, int R>
__global__ void __launch_bounds__(kThreads) step2d_persistent(const __grid_constant__ PersistParams pp)
{
    extern __shared__ __align__(1024) float sm[];
    __shared__ uint64_t bar;
    const int ntiles = pp.base.tiles_x * pp.base.tiles_y;
    for (int n = 0; n < pp.nt; ++n) {
        const StepView v(pp, n);
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x)
            step2d_tile<SHAPE, M, 0, kModeForward, R>(v, t, sm, bar);
        if (n + 1 < pp.nt && !grid_sync(pp)) return;
    }
}

// Generic runtime-shape 2D kernel (any shape, 1 <= M <= kMaxM): scalar
// shared-memory reads, one row per thread (R = 1).
template <int MODE>
__global__ void __launch_bounds__(kThreads) step2d_generic(const __grid_constant__ StepParams p,
                                                           int shape, int M, int N)
{
    const int HX = round4(M);
    const int SW = kTX + 2 * HX;
    const int SH = kTZ + 2 * M;
    extern __shared__ __align__(1024) float sm[];
    __shared__ uint64_t bar;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int tile = blockIdx.x;
    const int x0 = (tile % p.tiles_x) * kTX;
    const int z0 = (tile / p.tiles_x) * kTZ;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, SW * SH * 4);
        tma_load_2d(sm, p.tmap, &bar, x0 - HX, z0 - M);
    }
    const int ib = p.inj_ptr ? p.inj_ptr[tile] : 0, ie = p.inj_ptr ? p.inj_ptr[tile + 1] : 0;
    const int sb = p.smp_ptr ? p.smp_ptr[tile] : 0, se = p.smp_ptr ? p.smp_ptr[tile + 1] : 0;
    const bool ok = mbar_wait_bounded(&bar, 0);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
            atomicOr(p.status, kStatusTimeout);
            mbar_wait_bounded(&bar, 0);
        }
        return;
    }
    const int xg = x0 + 4 * tx, zg = z0 + ty;
    const bool live = xg < p.nx && zg < p.nz;
    const int zl = M + ty;
    float o[4], dv[4], kk[4], uu[4], gm[4];
    const int64_t off = (int64_t)zg * p.pitch + xg;
    const float4 up = live ? ldg4(p.u_prev + off) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 kp = live ? ldg4(p.kappa + off) : make_float4(0.f, 0.f, 0.f, 0.f);
    uu[0] = up.x; uu[1] = up.y; uu[2] = up.z; uu[3] = up.w;
    kk[0] = kp.x; kk[1] = kp.y; kk[2] = kp.z; kk[3] = kp.w;
    const float d2z = layer_d2(zg, p.phys_lo[2], p.phys_hi[2]);
    for (int j = 0; j < 4; ++j) {
        const int xc = HX + 4 * tx + j;
        // centre-free Laplacian (see step2d_tile)
        const float c = sm[zl * SW + xc];
        const float u2 = c + c, u4 = u2 + u2;
        float lap = 0.f;
        for (int q = 0; q <= M; ++q) {
            const int E = shape_ext(shape, M, N, q);
            if (E < 0) continue;
            const float *rp = sm + (zl + q) * SW + xc;
            const float *rm = sm + (zl - q) * SW + xc;
            float acc = q ? p.w[q] * ((rp[0] + rm[0]) - u2) : 0.f;
            for (int pp = 1; pp <= E; ++pp) {
                float s = rp[pp] + rp[-pp];
                if (q) s += rm[pp] + rm[-pp];
                acc = fmaf(p.w[pp * kWDim + q], s - (q ? u4 : u2), acc);
            }
            lap += acc;
        }
        gm[j] = sponge_g(p.gcoef, layer_d2(xg + j, p.phys_lo[0], p.phys_hi[0]) + d2z);
        dv[j] = step_update(c, uu[j], kk[j], lap, gm[j], o[j]);
    }
    float4 br = make_float4(o[0], o[1], o[2], o[3]);
    if (ib < ie)
        for_row(p.inj, ib, ie, zg, tx, [&](int j, const PtEntry &en) {
            float a = src_term(en.scale, p.inj_series[(int64_t)p.step * p.inj_ncol + en.col]);
            if (MODE == kModeAdjoint) a = __fmul_rn(a, kk[j]);
            add4(br, j, a);
        });
    o[0] = br.x; o[1] = br.y; o[2] = br.z; o[3] = br.w;
    for (int j = 0; j < 4; ++j)
        o[j] = sponge_div(o[j], gm[j]);
    const float4 un = make_float4(o[0], o[1], o[2], o[3]);
    if (sb < se)
        for_row(p.smp, sb, se, zg, tx, [&](int j, const PtEntry &en) {
            float v = get4(un, j) * en.scale;
            if (MODE == kModeAdjoint) v /= kk[j];
            p.smp_out[(int64_t)p.step * p.smp_ncol + en.col] = v;
        });
    if (!live) return;
    if (p.check) check_growth(p.status, un);
    *reinterpret_cast<float4 *>(p.u_prev + off) = un;
    if (MODE != kModeAdjoint && p.dseg_out)
        *reinterpret_cast<float4 *>(p.dseg_out + off) = make_float4(dv[0], dv[1], dv[2], dv[3]);
    if (MODE == kModeAdjoint) {
        const float4 d = ldg4(p.dseg_in + off);
        float4 g = *reinterpret_cast<float4 *>(p.gacc + off);
        g.x = fmaf(un.x, d.x, g.x); g.y = fmaf(un.y, d.y, g.y);
        g.z = fmaf(un.z, d.z, g.z); g.w = fmaf(un.w, d.w, g.w);
        *reinterpret_cast<float4 *>(p.gacc + off) = g;
    }
}

using KernelFn = void (*)(const StepParams);

template <int SHAPE, int M, int R>
KernelFn pick_mode(int mode)
{
    switch (mode) {
    case kModeForward: return step2d_kernel<SHAPE, M, 0, kModeForward, R>;
    case kModeStoreD: return step2d_kernel<SHAPE, M, 0, kModeForward, R>;
    default: return step2d_kernel<SHAPE, M, 0, kModeAdjoint, R>;
    }
}

// Specialised (shape, M, R) triples; everything else runs the generic kernel.
KernelFn lookup_fast(int shape, int M, int R, int mode)
{
#define FDW_C(S, MM, RR) \
    if (shape == S && M == MM && R == RR) return pick_mode<S, MM, RR>(mode);
    FDW_C(FD_CROSS, 2, 1) FDW_C(FD_CROSS, 4, 1) FDW_C(FD_CROSS, 8, 1)
    FDW_C(FD_CROSS, 2, 2) FDW_C(FD_CROSS, 4, 2) FDW_C(FD_CROSS, 8, 2)
    FDW_C(FD_CROSS, 2, 4) FDW_C(FD_CROSS, 4, 4) FDW_C(FD_CROSS, 8, 4)
    FDW_C(FD_RHOMBUS, 2, 2) FDW_C(FD_RHOMBUS, 4, 2) FDW_C(FD_RHOMBUS, 8, 2)
    FDW_C(FD_RHOMBUS, 2, 4) FDW_C(FD_RHOMBUS, 4, 4) FDW_C(FD_RHOMBUS, 8, 4)
    FDW_C(FD_SQUARE, 2, 2) FDW_C(FD_SQUARE, 4, 2) FDW_C(FD_SQUARE, 8, 2)
    FDW_C(FD_SQUARE, 2, 4) FDW_C(FD_SQUARE, 4, 4) FDW_C(FD_SQUARE, 8, 4)
#undef FDW_C
    return nullptr;
}

using BatchFn = void (*)(const BatchParams);

template <int S, int MM, int RR, int MODE>
BatchFn pick_batched_m(bool check)
{
    return check ? step2d_batched<S, MM, RR, MODE, true> : step2d_batched<S, MM, RR, MODE, false>;
}

// the growth check is compile-time (a run-time test in the store loop measured
// 1.2 % slower on the 48-shot batch)
template <int S, int MM, int RR>
BatchFn pick_batched(int mode, bool check)
{
    switch (mode) {
    case kModeForward: return pick_batched_m<S, MM, RR, kModeForward>(check);
    case kModeStoreD: return pick_batched_m<S, MM, RR, kModeStoreD>(check);
    default: return pick_batched_m<S, MM, RR, kModeAdjoint>(check);
    }
}

BatchFn lookup_batched(int shape, int M, int R, int mode = kModeForward, bool check = false)
{
#define FDW_B(S, MM, RR) \
    if (shape == S && M == MM && R == RR) return pick_batched<S, MM, RR>(mode, check);
    FDW_B(FD_CROSS, 2, 2) FDW_B(FD_CROSS, 4, 2) FDW_B(FD_CROSS, 8, 2)
    FDW_B(FD_CROSS, 2, 4) FDW_B(FD_CROSS, 4, 4) FDW_B(FD_CROSS, 8, 4)
#undef FDW_B
    return nullptr;
}

using PersistFn = void (*)(const PersistParams);

PersistFn lookup_persist(int shape, int M, int R)
{
#define FDW_P(S, MM, RR) \
    if (shape == S && M == MM && R == RR) return step2d_persistent<S, MM, RR>;
    FDW_P(FD_CROSS, 2, 1) FDW_P(FD_CROSS, 4, 1) FDW_P(FD_CROSS, 8, 1)
    FDW_P(FD_CROSS, 2, 2) FDW_P(FD_CROSS, 4, 2) FDW_P(FD_CROSS, 8, 2)
    FDW_P(FD_CROSS, 2, 4) FDW_P(FD_CROSS, 4, 4) FDW_P(FD_CROSS, 8, 4)
    FDW_P(FD_RHOMBUS, 2, 2) FDW_P(FD_RHOMBUS, 4, 2) FDW_P(FD_RHOMBUS, 8, 2)
    FDW_P(FD_RHOMBUS, 2, 4) FDW_P(FD_RHOMBUS, 4, 4) FDW_P(FD_RHOMBUS, 8, 4)
    FDW_P(FD_SQUARE, 2, 2) FDW_P(FD_SQUARE, 4, 2) FDW_P(FD_SQUARE, 8, 2)
    FDW_P(FD_SQUARE, 2, 4) FDW_P(FD_SQUARE, 4, 4) FDW_P(FD_SQUARE, 8, 4)
#undef FDW_P
    return nullptr;
}

}  // namespace

// Resident CTAs of the persistent 2D kernel for this variant (0: not available).
int persist2d_grid(const Variant &v, int ntiles)
{
    PersistFn fn = lookup_persist(v.shape, v.M, v.tz / kTZ);
    if (!fn || v.generic) return 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem) != cudaSuccess)
        return 0;
    int dev = 0, nsm = 0, per = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (!coop || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kThreads, v.smem) != cudaSuccess)
        return 0;
    const int g = per * nsm;
    return g < ntiles ? g : ntiles;
}

cudaError_t launch_persist2d(const Variant &v, const PersistParams &pp, int grid, cudaStream_t s)
{
    PersistFn fn = lookup_persist(v.shape, v.M, v.tz / kTZ);
    if (!fn) return cudaErrorInvalidValue;
    void *args[] = {const_cast<PersistParams *>(&pp)};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(fn), dim3(grid), dim3(kThreads),
                                       args, v.smem, s);
}

template <int R>
size_t batch_smem(int M)
{
    return M == 2 ? StreamCfg<2, R>::SMEM : M == 4 ? StreamCfg<4, R>::SMEM : StreamCfg<8, R>::SMEM;
}

int batch2d_variants(int shape, int M, int *r_out, int cap)
{
    int n = 0;
    for (int r : {2, 4})
        if (n < cap && lookup_batched(shape, M, r)) r_out[n++] = r;
    return n;
}

int batch2d_variant(int shape, int M, int64_t total_tiles4, Variant *v, int r_pref)
{
    // default 64 x 32 tiles (R = 2): small slots, so each CTA keeps several
    // tiles of copies in flight while it computes one; 64 x 64 (R = 4) has
    // less halo per point and fewer, larger copies
    const int R = r_pref > 0 ? r_pref : 2;
    (void)total_tiles4;
    if (!lookup_batched(shape, M, R)) return FD_ERR_UNSUPPORTED;
    v->dim = 2;
    v->shape = shape;
    v->M = M;
    v->N = 0;
    v->generic = 0;
    v->threads = kThreads + 32;
    v->tx = kTX;
    v->tz = kTZ * R;
    v->box[0] = kTX + 2 * round4(M);
    v->box[1] = kTZ * R + 2 * M;
    v->box[2] = 1;
    v->tbox[0] = kTX;
    v->tbox[1] = kTZ * R;
    v->smem = R == 4 ? batch_smem<4>(M) : batch_smem<2>(M);
    return FD_OK;
}

cudaError_t launch_batched2d(const Variant &v, const BatchParams &bp, int ntiles, cudaStream_t s,
                             int mode)
{
    BatchFn fn = lookup_batched(v.shape, v.M, v.tz / kTZ, mode, bp.check != 0);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
    if (e != cudaSuccess) return e;
    if (ntiles <= 0) return cudaSuccess;
    // persistent CTAs: as many as are resident at once, at most one per tile
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, v.threads, v.smem)) != cudaSuccess)
        return e;
    const int grid = std::min(ntiles, std::max(1, per_sm) * sms);
    fn<<<grid, v.threads, v.smem, s>>>(bp);
    return cudaGetLastError();
}

using BatchPFn = void (*)(const BatchParams, int);

BatchPFn lookup_batched_persistent(int shape, int M, int R)
{
#define FDW_B(S, MM, RR) \
    if (shape == S && M == MM && R == RR) return step2d_batched_persistent<S, MM, RR>;
    FDW_B(FD_CROSS, 2, 2) FDW_B(FD_CROSS, 4, 2) FDW_B(FD_CROSS, 8, 2)
    FDW_B(FD_CROSS, 2, 4) FDW_B(FD_CROSS, 4, 4) FDW_B(FD_CROSS, 8, 4)
#undef FDW_B
    return nullptr;
}

using Batch2Fn = void (*)(const BatchParams);

Batch2Fn lookup_batched2(int shape, int M)
{
    if (shape == FD_CROSS && M == 2) return step2d_batched2<FD_CROSS, 2, 2>;
    if (shape == FD_CROSS && M == 4) return step2d_batched2<FD_CROSS, 4, 2>;
    return nullptr;
}

template <int M>
void fill_geo2(Batch2Geo *g, size_t *smem)
{
    using C = Stream2Cfg<M, 2>;
    g->tz = C::TZ;
    g->hx = C::HX;
    g->hxc = C::HXC;
    g->cbox[0] = C::CW; g->cbox[1] = C::CH;
    g->pbox[0] = C::EW; g->pbox[1] = C::EH;
    *smem = C::SMEM;
}

int batch2d2_geometry(int shape, int M, Batch2Geo *g)
{
    if (!lookup_batched2(shape, M)) return FD_ERR_UNSUPPORTED;
    size_t smem;
    if (M == 2) fill_geo2<2>(g, &smem);
    else fill_geo2<4>(g, &smem);
    return FD_OK;
}

cudaError_t launch_batched2d2(const Variant &v, const BatchParams &bp, int ntiles, cudaStream_t s)
{
    Batch2Fn fn = lookup_batched2(v.shape, v.M);
    if (!fn) return cudaErrorInvalidValue;
    Batch2Geo g;
    size_t smem = 0;
    if (v.M == 2) fill_geo2<2>(&g, &smem);
    else fill_geo2<4>(&g, &smem);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (ntiles <= 0) return cudaSuccess;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads + 32, smem)) != cudaSuccess)
        return e;
    const int grid = std::min(ntiles, std::max(1, per_sm) * sms);
    fn<<<grid, kThreads + 32, smem, s>>>(bp);
    return cudaGetLastError();
}

cudaError_t launch_batched2d_persistent(const Variant &v, const BatchParams &bp, int ntiles, int nt,
                                       cudaStream_t s)
{
    BatchPFn fn = lookup_batched_persistent(v.shape, v.M, v.tz / kTZ);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
    if (e != cudaSuccess) return e;
    if (ntiles <= 0 || nt <= 0) return cudaSuccess;
    int dev = 0, sms = 0, per_sm = 0, coop = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess) return e;
    if (!coop) return cudaErrorNotSupported;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, v.threads, v.smem)) != cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = std::min(ntiles, per_sm * sms);   // all resident: the grid barrier needs it
    void *args[] = {const_cast<BatchParams *>(&bp), &nt};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(fn), dim3(grid), dim3(v.threads), args,
                                       v.smem, s);
}

int variants_2d(int shape, int M, int *r_out, int cap)
{
    int n = 0;
    for (int r : {4, 2, 1})
        if (n < cap && lookup_fast(shape, M, r, 0)) r_out[n++] = r;
    return n;
}

int select_variant_2d(int shape, int M, int N, int64_t nx, int64_t nz, Variant *v, int r_pref)
{
    v->dim = 2;
    v->shape = shape;
    v->M = M;
    v->N = N;
    v->threads = kThreads;
    v->tx = kTX;
    // R rows per thread: the preferred R when it is compiled, else the largest
    // compiled R whose tiles still fill the GPU (two CTAs per SM on 152 SMs),
    // else the smallest compiled R; the generic kernel runs R = 1.
    auto tiles = [&](int r) {
        return ((nx + kTX - 1) / kTX) * ((nz + r * kTZ - 1) / (r * kTZ));
    };
    int R = r_pref > 0 && lookup_fast(shape, M, r_pref, 0) ? r_pref : 0;
    for (int r : {4, 2, 1})
        if (!R && lookup_fast(shape, M, r, 0) && tiles(r) >= 2 * 152) R = r;
    for (int r : {1, 2, 4})
        if (!R && lookup_fast(shape, M, r, 0)) R = r;
    v->generic = R ? 0 : 1;
    if (v->generic) R = 1;
    v->tz = kTZ * R;
    const int HX = round4(M);
    v->box[0] = kTX + 2 * HX;
    v->box[1] = kTZ * R + 2 * M;
    v->box[2] = 1;
    v->smem = (size_t)v->box[0] * v->box[1] * sizeof(float);
    return 0;
}

cudaError_t launch_step2d(const Variant &v, int mode, const StepParams &p, cudaStream_t s)
{
    const int ntiles = p.tiles_x * p.tiles_y;
    if (ntiles <= 0) return cudaSuccess;
    if (!v.generic) {
        KernelFn fn = lookup_fast(v.shape, v.M, v.tz / kTZ, mode);
        if (!fn) return cudaErrorInvalidValue;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)v.smem);
        if (e != cudaSuccess) return e;
        fn<<<ntiles, kThreads, v.smem, s>>>(p);
        return cudaGetLastError();
    }
    void (*fn)(const StepParams, int, int, int) =
        mode == kModeForward ? step2d_generic<kModeForward>
        : mode == kModeStoreD ? step2d_generic<kModeForward> : step2d_generic<kModeAdjoint>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)v.smem);
    if (e != cudaSuccess) return e;
    fn<<<ntiles, kThreads, v.smem, s>>>(p, v.shape, v.M, v.N);
    return cudaGetLastError();
}

}  // namespace fdw
