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
// outputs it touches).
#include "step3d_common.cuh"

namespace fdw {

namespace {




// ---------------------------------------------------------------------------
// Cross stencils: warp-specialised TMA pipeline, z-arm in a register queue.
//
// One producer warp streams, for every plane z of the chunk, one ring slot
// holding: the u_cur plane with its x/y halo (x and y arms, centre), the
// u_prev and kappa tiles of plane z, and the u_cur tile of plane z+M (the
// newest entry of the z-arm queue).  Slots are guarded by a full and an empty
// mbarrier each, so consumer warps run ahead of one another by up to the
// ring depth; there is no block-wide barrier in the plane loop.  Consumers
// keep the 2M+1 centre values of their column in a register queue; the loop
// is unrolled by the queue length so queue indices are compile-time.  The
// first 2M slots of a chunk carry only queue entries (planes zb-M .. zb+M-1).
// Every wait is bounded; on a time-out the block sets the status bit, the
// producer waits (bounded) for its copies in flight, and the block returns.
// ---------------------------------------------------------------------------
template <int M, int TY>
struct CrossCfg {
    static constexpr int HX = round4(M);
    static constexpr int PW = kTX3 + 2 * HX;
    static constexpr int PH = TY + 2 * M;
    static constexpr int AEL = (PW * PH + 31) & ~31;      // halo plane (floats, padded)
    static constexpr int TEL = kTX3 * TY;                 // tile (floats, multiple of 32)
    static constexpr int SLOT = AEL + 3 * TEL;            // A | u_prev | kappa | queue tile
    static constexpr int MINB = ctas_per_sm(true, M, TY);
    static constexpr int NR = ring_depth(SLOT, MINB);
    static constexpr int NCW = TY / 2;                    // consumer warps
    static constexpr int THREADS = 16 * TY + 32;
};

template <int M, int MODE, int TY, bool CHECK>
__global__ void __launch_bounds__(CrossCfg<M, TY>::THREADS, CrossCfg<M, TY>::MINB)
step3d_cross(const __grid_constant__ StepParams p)
{
    using C = CrossCfg<M, TY>;
    constexpr int HX = C::HX, PW = C::PW, PH = C::PH;
    constexpr int NR = C::NR, SLOT = C::SLOT;
    constexpr int QL = 2 * M + 1;
    constexpr uint32_t BYTES_FULL = (PW * PH + 3 * C::TEL) * 4;
    constexpr uint32_t BYTES_Q = C::TEL * 4;
    extern __shared__ __align__(1024) float sm[];
    __shared__ uint64_t full[NR], empty[NR];
    __shared__ int abort_flag;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int ntile = p.tiles_x * p.tiles_y;
    const int tile = blockIdx.x % ntile, zc = blockIdx.x / ntile;
    const int x0 = (tile % p.tiles_x) * kTX3, y0 = (tile / p.tiles_x) * TY;
    const int zb = zc * p.zchunk;
    const int nz = (int)p.nz;
    const int ze = min(nz, zb + p.zchunk);
    const int L = ze - zb;            // planes computed
    const int S = L + 2 * M;          // slots streamed (the first 2M carry queue tiles only)

    if (tid == 0) {
        for (int i = 0; i < NR; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], C::NCW);
        }
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == C::NCW) {
        // ------------------------------ producer ------------------------------
        if (lane != 0) return;
        prefetch_tmap(p.tmap);
        prefetch_tmap(p.tmap_cur_t);
        prefetch_tmap(p.tmap_prev_t);
        prefetch_tmap(p.tmap_kappa_t);
        volatile int *abort_v = &abort_flag;
        int slot = 0;
        int s = 0;
        for (; s < S; ++s) {
            // reuse of a slot waits for the consumers' release of stream index s - NR,
            // i.e. the completion of empty phase s / NR - 1
            if (s >= NR && !mbar_wait_bounded(&empty[slot], (uint32_t)((s / NR - 1) & 1), p.wait_cycles)) {
                atomicOr(p.status, kStatusTimeout);
                *abort_v = 1;
                break;
            }
            if (*abort_v) break;
            // test hook: CTA 0 issues nothing for slot drop_slot, so its consumers' wait runs out
            if (blockIdx.x == 0 && s == p.drop_slot) {
                if (++slot == NR) slot = 0;
                continue;
            }
            float *dst = sm + slot * SLOT;
            const int zq = zb + s - M;                  // queue plane carried by this slot
            if (s < 2 * M) {
                mbar_arrive_expect_tx(&full[slot], BYTES_Q);
            } else {
                const int z = zb + s - 2 * M;
                mbar_arrive_expect_tx(&full[slot], BYTES_FULL);
                tma_load_3d(dst, p.tmap, &full[slot], x0 - HX, y0 - M, z);
                tma_load_3d(dst + C::AEL, p.tmap_prev_t, &full[slot], x0, y0, z);
                tma_load_3d(dst + C::AEL + C::TEL, p.tmap_kappa_t, &full[slot], x0, y0, z);
            }
            tma_load_3d(dst + C::AEL + 2 * C::TEL, p.tmap_cur_t, &full[slot], x0, y0, zq);
            if (++slot == NR) slot = 0;
        }
        if (*abort_v) {   // let copies already issued land before the block exits
            for (int i = max(0, s - NR); i < s; ++i)
                if (!(blockIdx.x == 0 && i == p.drop_slot))
                    mbar_wait_bounded(&full[i % NR], (i / NR) & 1, 100000000LL);
        }
        return;
    }

    // ------------------------------- consumers --------------------------------
    const int ty = tid >> 4, tx = tid & 15;
    const int xg = x0 + 4 * tx, yg = y0 + ty;
    const bool colok = xg < p.nx && yg < p.ny;
    const int64_t colo = (int64_t)yg * p.pitch + xg;
    float d2xy[4];
    {
        const float d2y = layer_d2(yg, p.phys_lo[1], p.phys_hi[1]);
#pragma unroll
        for (int j = 0; j < 4; ++j) d2xy[j] = layer_d2(xg + j, p.phys_lo[0], p.phys_hi[0]) + d2y;
    }
    int ki = p.inj_ptr ? p.inj_ptr[tile] : 0, kie = p.inj_ptr ? p.inj_ptr[tile + 1] : 0;
    int ks = p.smp_ptr ? p.smp_ptr[tile] : 0, kse = p.smp_ptr ? p.smp_ptr[tile + 1] : 0;
    int zinj = ki < kie ? p.inj[ki].z : 0x7fffffff;    // z of the next table entry
    int zsmp = ks < kse ? p.smp[ks].z : 0x7fffffff;
    const int cA = (M + ty) * PW + HX + 4 * tx;        // my centre in the halo plane
    const int cT = ty * kTX3 + 4 * tx;                 // my element in a tile

    // Queue of centre values as packed pairs (x, y) and (z, w).  Unrolled
    // (M <= 4): the plane fed at stream index s sits in slot s mod QL and the
    // loop is unrolled by QL.  Blocked (M >= 6, smaller code): the loop is
    // unrolled by UF = 3 over a queue of QL + 2 slots that moves down UF slots
    // at the start of each block; sub-step uu feeds slot QL-1+uu.  (Either
    // form for either M measured within 0.2 % of the other on the 460^3 grid.)
    constexpr bool kUnroll = M <= 4;
    constexpr int UF = kUnroll ? QL : 3;
    constexpr int QN = kUnroll ? QL : QL + UF - 1;
    f32x2 qa[QN], qb[QN];
#pragma unroll
    for (int i = 0; i < QN; ++i) qa[i] = qb[i] = 0ull;
    int slot = 0;
    uint32_t fph = 0;
    bool ok = true;

    for (int k0 = 0; k0 < S; k0 += UF) {
        if (!kUnroll) {
#pragma unroll
            for (int i = 0; i < QN - UF; ++i) {
                qa[i] = qa[i + UF];
                qb[i] = qb[i + UF];
            }
        }
#pragma unroll
        for (int uu = 0; uu < UF; ++uu) {
            const int si = k0 + uu;            // 0-based stream index
            if (si >= S) break;
            const int u = kUnroll ? uu : QL - 1 + uu;   // slot of the plane fed now
            ok = ok && mbar_wait_bounded(&full[slot], fph, p.wait_cycles);
            if (!ok) break;
            const float *P = sm + slot * SLOT;
            ld4x2(P + C::AEL + 2 * C::TEL + cT, qa[u], qb[u]);   // plane zb + si - M
            if (si >= 2 * M) {
                const int z = zb + si - 2 * M;
                // queue slot of plane z + d: (u - M + d) mod QL unrolled, uu + M + d blocked
                float win[4 + 2 * HX];
#pragma unroll
                for (int i = 0; i < (4 + 2 * HX) / 4; ++i) {
                    const float4 a = ld4(P + cA - HX + 4 * i);
                    win[4 * i] = a.x; win[4 * i + 1] = a.y; win[4 * i + 2] = a.z; win[4 * i + 3] = a.w;
                }
                // centre-free Laplacian: W[0][m] ((sum of the 6 points at distance
                // m) - 6 u), the six summed as x pair + (y pair + z pair) so that a
                // constant field gives 6u rounded exactly like the 6u subtracted
                const f32x2 c01 = pk2(win[HX], win[HX + 1]), c23 = pk2(win[HX + 2], win[HX + 3]);
                const f32x2 u2_01 = add2(c01, c01), u2_23 = add2(c23, c23);
                const f32x2 u6_01 = add2(u2_01, add2(u2_01, u2_01));
                const f32x2 u6_23 = add2(u2_23, add2(u2_23, u2_23));
                f32x2 l01 = 0ull, l23 = 0ull;
#pragma unroll
                for (int m = 1; m <= M; ++m) {
                    f32x2 a01, a23, b01, b23;
                    ld4x2(P + cA + m * PW, a01, a23);
                    ld4x2(P + cA - m * PW, b01, b23);
                    const int ip = kUnroll ? (u - M + m + 2 * QL) % QL : uu + M + m;
                    const int im = kUnroll ? (u - M - m + 2 * QL) % QL : uu + M - m;
                    const f32x2 wm = p.w2[m];
                    const f32x2 x01 = pk2(win[HX + m] + win[HX - m], win[HX + 1 + m] + win[HX + 1 - m]);
                    const f32x2 x23 = pk2(win[HX + 2 + m] + win[HX + 2 - m], win[HX + 3 + m] + win[HX + 3 - m]);
                    const f32x2 s01 = add2(x01, add2(add2(a01, b01), add2(qa[ip], qa[im])));
                    const f32x2 s23 = add2(x23, add2(add2(a23, b23), add2(qb[ip], qb[im])));
                    l01 = fma2(wm, sub2(s01, u6_01), l01);
                    l23 = fma2(wm, sub2(s23, u6_23), l23);
                }
                f32x2 up01, up23, k01, k23;
                ld4x2(P + C::AEL + cT, up01, up23);
                ld4x2(P + C::AEL + C::TEL + cT, k01, k23);
                // the slot has been read: release it to the producer
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[slot]);
                const int ic = kUnroll ? (u - M + 2 * QL) % QL : uu + M;
                const float d2z = layer_d2(z, p.phys_lo[2], p.phys_hi[2]);
                float g[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) g[j] = sponge_g(p.gcoef, d2xy[j] + d2z);
                f32x2 o01, o23;
                const f32x2 dv01 = step_update2(qa[ic], up01, k01, l01, pk2(g[0], g[1]), o01);
                const f32x2 dv23 = step_update2(qb[ic], up23, k23, l23, pk2(g[2], g[3]), o23);
                float4 o, kk;
                upk2(o01, o.x, o.y);
                upk2(o23, o.z, o.w);
                upk2(k01, kk.x, kk.y);
                upk2(k23, kk.z, kk.w);
                if (z >= zinj) {
                    const InjOut r = inject_plane<MODE>(p, ki, kie, z, tx, ty, o, kk);
                    o = r.o;
                    ki = r.k;
                    zinj = r.z;
                }
                if (g[0] != 0.f || g[1] != 0.f || g[2] != 0.f || g[3] != 0.f) {
                    o.x = sponge_div(o.x, g[0]);
                    o.y = sponge_div(o.y, g[1]);
                    o.z = sponge_div(o.z, g[2]);
                    o.w = sponge_div(o.w, g[3]);
                }
                if (z >= zsmp) {
                    const int2 r = sample_plane<MODE>(p, ks, kse, z, tx, ty, o, kk);
                    ks = r.x;
                    zsmp = r.y;
                }
                if (colok) {
                    const int64_t off = (int64_t)z * p.plane + colo;
                    if (CHECK) check_growth(p.status, o);
                    *reinterpret_cast<float4 *>(p.u_prev + off) = o;
                    if (MODE == kModeStoreD)
                        *reinterpret_cast<ulonglong2 *>(p.dseg_out + off) = make_ulonglong2(dv01, dv23);
                    if (MODE == kModeAdjoint) {
                        const float4 dd = ldg4(p.dseg_in + off);
                        float4 ga = *reinterpret_cast<float4 *>(p.gacc + off);
                        ga.x = fmaf(o.x, dd.x, ga.x); ga.y = fmaf(o.y, dd.y, ga.y);
                        ga.z = fmaf(o.z, dd.z, ga.z); ga.w = fmaf(o.w, dd.w, ga.w);
                        *reinterpret_cast<float4 *>(p.gacc + off) = ga;
                    }
                }
            } else {
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[slot]);
            }
            if (++slot == NR) {
                slot = 0;
                fph ^= 1u;
            }
        }
        if (!ok) break;
    }
    if (!ok) {
        atomicOr(p.status, kStatusTimeout);
        *reinterpret_cast<volatile int *>(&abort_flag) = 1;
    }
}

template <int M, int TY>
struct PlanarCfg {
    static constexpr int HX = round4(M);
    static constexpr int PW = kTX3 + 2 * HX;
    static constexpr int PH = TY + 2 * M;
    static constexpr int AEL = (PW * PH + 31) & ~31;
    static constexpr int TEL = kTX3 * TY;
    static constexpr int SLOT = AEL + 3 * TEL;            // A | u_cur(P-M) | u_prev | kappa
    static constexpr int MINB = ctas_per_sm(false, M, TY);
    static constexpr int NR = ring_depth(SLOT, MINB);
    static constexpr int NCW = TY / 2;
    static constexpr int THREADS = 16 * TY + 32;
};

template <int SHAPE, int M, int MODE, int TY, bool CHECK>
__global__ void __launch_bounds__(PlanarCfg<M, TY>::THREADS, PlanarCfg<M, TY>::MINB)
step3d_planar(const __grid_constant__ StepParams p)
{
    using C = PlanarCfg<M, TY>;
    constexpr int HX = C::HX, PW = C::PW, PH = C::PH;
    constexpr int NR = C::NR, SLOT = C::SLOT;
    constexpr int QL = 2 * M + 1;
    constexpr uint32_t BYTES_FULL = (PW * PH + 3 * C::TEL) * 4;
    constexpr uint32_t BYTES_A = PW * PH * 4;
    extern __shared__ __align__(1024) float sm[];
    __shared__ uint64_t full[NR], empty[NR];
    __shared__ int abort_flag;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int ntile = p.tiles_x * p.tiles_y;
    const int tile = blockIdx.x % ntile, zc = blockIdx.x / ntile;
    const int x0 = (tile % p.tiles_x) * kTX3, y0 = (tile / p.tiles_x) * TY;
    const int zb = zc * p.zchunk;
    const int nz = (int)p.nz;
    const int ze = min(nz, zb + p.zchunk);
    const int L = ze - zb;
    const int S = L + 2 * M;          // planes zb-M .. ze+M-1

    if (tid == 0) {
        for (int i = 0; i < NR; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], C::NCW);
        }
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == C::NCW) {
        if (lane != 0) return;
        prefetch_tmap(p.tmap);
        prefetch_tmap(p.tmap_cur_t);
        prefetch_tmap(p.tmap_prev_t);
        prefetch_tmap(p.tmap_kappa_t);
        volatile int *abort_v = &abort_flag;
        int slot = 0, t = 0;
        for (; t < S; ++t) {
            if (t >= NR && !mbar_wait_bounded(&empty[slot], (uint32_t)((t / NR - 1) & 1), p.wait_cycles)) {
                atomicOr(p.status, kStatusTimeout);
                *abort_v = 1;
                break;
            }
            if (*abort_v) break;
            // test hook: CTA 0 issues nothing for slot drop_slot, so its consumers' wait runs out
            if (blockIdx.x == 0 && t == p.drop_slot) {
                if (++slot == NR) slot = 0;
                continue;
            }
            float *dst = sm + slot * SLOT;
            const int P = zb - M + t;
            if (t < 2 * M) {
                mbar_arrive_expect_tx(&full[slot], BYTES_A);
            } else {
                const int z = P - M;
                mbar_arrive_expect_tx(&full[slot], BYTES_FULL);
                tma_load_3d(dst + C::AEL, p.tmap_cur_t, &full[slot], x0, y0, z);
                tma_load_3d(dst + C::AEL + C::TEL, p.tmap_prev_t, &full[slot], x0, y0, z);
                tma_load_3d(dst + C::AEL + 2 * C::TEL, p.tmap_kappa_t, &full[slot], x0, y0, z);
            }
            tma_load_3d(dst, p.tmap, &full[slot], x0 - HX, y0 - M, P);
            if (++slot == NR) slot = 0;
        }
        if (*abort_v) {
            for (int i = max(0, t - NR); i < t; ++i)
                if (!(blockIdx.x == 0 && i == p.drop_slot))
                    mbar_wait_bounded(&full[i % NR], (i / NR) & 1, 100000000LL);
        }
        return;
    }

    const int ty = tid >> 4, tx = tid & 15;
    const int xg = x0 + 4 * tx, yg = y0 + ty;
    const bool colok = xg < p.nx && yg < p.ny;
    const int64_t colo = (int64_t)yg * p.pitch + xg;
    float d2xy[4];
    {
        const float d2y = layer_d2(yg, p.phys_lo[1], p.phys_hi[1]);
#pragma unroll
        for (int j = 0; j < 4; ++j) d2xy[j] = layer_d2(xg + j, p.phys_lo[0], p.phys_hi[0]) + d2y;
    }
    int ki = p.inj_ptr ? p.inj_ptr[tile] : 0, kie = p.inj_ptr ? p.inj_ptr[tile + 1] : 0;
    int ks = p.smp_ptr ? p.smp_ptr[tile] : 0, kse = p.smp_ptr ? p.smp_ptr[tile + 1] : 0;
    const int cA = (M + ty) * PW + HX + 4 * tx;
    const int cT = ty * kTX3 + 4 * tx;

    int zinj = ki < kie ? p.inj[ki].z : 0x7fffffff;
    int zsmp = ks < kse ? p.smp[ks].z : 0x7fffffff;
    // acc[i] holds output P - M + i after the shift at plane P (i = 0..2M); the
    // accumulators move down one slot per plane (no unroll: small code)
    // acc[uu + i][h] holds lanes (2h, 2h+1) of output P - M + i at sub-step uu
    // of a block of UF planes (i = 0..2M); at the start of each block the
    // accumulators move down UF slots and the top UF slots (outputs that start
    // in this block) are cleared
    constexpr int UF = 3;
    constexpr int AN = QL + UF - 1;
    f32x2 acc[AN][2];
#pragma unroll
    for (int i = 0; i < AN; ++i) acc[i][0] = acc[i][1] = 0ull;
    // centre values of the previous plane; the first plane's step only feeds
    // outputs below the chunk, so its start value does not matter
    f32x2 cprev[2] = {0ull, 0ull};
    int slot = 0;
    uint32_t fph = 0;
    bool ok = true;

    for (int t0 = 0; t0 < S; t0 += UF) {
#pragma unroll
        for (int i = 0; i < AN; ++i) {
            acc[i][0] = i + UF < AN ? acc[i + UF][0] : 0ull;
            acc[i][1] = i + UF < AN ? acc[i + UF][1] : 0ull;
        }
#pragma unroll
        for (int uu = 0; uu < UF; ++uu) {
            const int t = t0 + uu;
            if (t >= S) break;
            ok = ok && mbar_wait_bounded(&full[slot], fph, p.wait_cycles);
            if (!ok) break;
            const float *A = sm + slot * SLOT;
            // Centre-free Laplacian, split per plane: T[s] sums the points of plane
            // P at |dz| = s minus plane P's own centre value c(P) (n points, n c(P)
            // subtracted before weighting); the z-axis remainder
            // sum_s A_s (c(z+s) + c(z-s) - 2 c(z)), A_s the total weight at |dz| = s,
            // is telescoped into plane-to-plane steps dl(P) = c(P) - c(P-1):
            // output P - s gets +B_s dl(P) (s >= 1) and output P + s gets
            // -B_{s+1} dl(P) (s >= 0), B_i = sum_{s >= i} A_s.  A constant field
            // gives exactly zero, and every accumulated term is a small difference.
            // Lanes (0,1) and (2,3) of the thread's float4 go two per instruction.
            f32x2 T[M + 1][2];
#pragma unroll
            for (int s = 0; s <= M; ++s) T[s][0] = T[s][1] = 0ull;
            f32x2 u2[2], u4[2], dl[2];
            {   // row y of P: in-plane x line (s = 0) and xz lines (s >= 1)
                float win[4 + 2 * HX];
#pragma unroll
                for (int i = 0; i < (4 + 2 * HX) / 4; ++i) {
                    const float4 a = ld4(A + cA - HX + 4 * i);
                    win[4 * i] = a.x; win[4 * i + 1] = a.y; win[4 * i + 2] = a.z; win[4 * i + 3] = a.w;
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int b = HX + 2 * h;
                    const f32x2 c = pk2(win[b], win[b + 1]);
                    dl[h] = sub2(c, cprev[h]);
                    cprev[h] = c;
                    u2[h] = add2(c, c);
                    u4[h] = add2(u2[h], u2[h]);
                    f32x2 ps[M + 1];
#pragma unroll
                    for (int pp = 1; pp <= M; ++pp)
                        ps[pp] = sub2(pair_add(win, b + pp, b - pp), u2[h]);
#pragma unroll
                    for (int s = 0; s <= M; ++s) {
                        const int E = shape_ext(SHAPE, M, 0, s);
                        if (E < 1) continue;
                        f32x2 a = mul2(p.w2[kW3 + s], ps[1]);
#pragma unroll
                        for (int pp = 2; pp <= E; ++pp)
                            a = fma2(p.w2[pp * kW3 + s], ps[pp], a);
                        T[s][h] = a;
                    }
                }
            }
#pragma unroll
            for (int q = 1; q <= M; ++q) {   // row pairs y +- q: in-plane rows and yz columns
                const int E = shape_ext(SHAPE, M, 0, q);
                const int E4 = round4(E);
                float win[4 + 2 * HX];
                const float *rp = A + cA + q * PW - E4;
                const float *rm = A + cA - q * PW - E4;
#pragma unroll
                for (int i = 0; i < (4 + 2 * E4) / 4; ++i) {
                    f32x2 a0, a1, b0, b1;
                    ld4x2(rp + 4 * i, a0, a1);
                    ld4x2(rm + 4 * i, b0, b1);
                    upk2(add2(a0, b0), win[4 * i], win[4 * i + 1]);
                    upk2(add2(a1, b1), win[4 * i + 2], win[4 * i + 3]);
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int b = E4 + 2 * h;
                    const f32x2 d0 = sub2(pk2(win[b], win[b + 1]), u2[h]);
                    f32x2 a = mul2(p.w2[q], d0);
#pragma unroll
                    for (int pp = 1; pp <= E; ++pp)
                        a = fma2(p.w2[pp * kW3 + q], sub2(pair_add(win, b + pp, b - pp), u4[h]), a);
                    T[0][h] = add2(T[0][h], a);
#pragma unroll
                    for (int s = 1; s <= M; ++s)
                        if (q <= shape_ext(SHAPE, M, 0, s))
                            T[s][h] = fma2(p.w2[q * kW3 + s], d0, T[s][h]);
                }
            }
            float4 cv = make_float4(0.f, 0.f, 0.f, 0.f), upv = cv, kpv = cv;
            const bool fin = t >= 2 * M;
            if (fin) {
                cv = ld4(A + C::AEL + cT);
                upv = ld4(A + C::AEL + C::TEL + cT);
                kpv = ld4(A + C::AEL + 2 * C::TEL + cT);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);
            if (++slot == NR) {
                slot = 0;
                fph ^= 1u;
            }
            // scatter: T[0] - B_1 dl -> output P (slot M); T[s] + B_s dl -> output
            // P - s; T[s] - B_{s+1} dl -> output P + s
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                acc[uu + M][h] = add2(acc[uu + M][h], fma2(p.zm2[0], dl[h], T[0][h]));
#pragma unroll
                for (int s = 1; s <= M; ++s) {
                    acc[uu + M - s][h] = add2(acc[uu + M - s][h],
                                              fma2(p.zp2[s], dl[h], T[s][h]));
                    const f32x2 tp = s < M ? fma2(p.zm2[s], dl[h], T[s][h])
                                           : T[s][h];
                    acc[uu + M + s][h] = add2(acc[uu + M + s][h], tp);
                }
            }
            if (!fin) continue;
            const int z = zb + t - 2 * M;             // output z = P - M is complete (slot 0)
            const float d2z = layer_d2(z, p.phys_lo[2], p.phys_hi[2]);
            float g[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) g[j] = sponge_g(p.gcoef, d2xy[j] + d2z);
            f32x2 o01, o23;
            const f32x2 dv01 = step_update2(pk2(cv.x, cv.y), pk2(upv.x, upv.y), pk2(kpv.x, kpv.y),
                                            acc[uu][0], pk2(g[0], g[1]), o01);
            const f32x2 dv23 = step_update2(pk2(cv.z, cv.w), pk2(upv.z, upv.w), pk2(kpv.z, kpv.w),
                                            acc[uu][1], pk2(g[2], g[3]), o23);
            float4 o;
            upk2(o01, o.x, o.y);
            upk2(o23, o.z, o.w);
            if (z >= zinj) {
                const InjOut r = inject_plane<MODE>(p, ki, kie, z, tx, ty, o, kpv);
                o = r.o;
                ki = r.k;
                zinj = r.z;
            }
            if (g[0] != 0.f || g[1] != 0.f || g[2] != 0.f || g[3] != 0.f) {
                o.x = sponge_div(o.x, g[0]);
                o.y = sponge_div(o.y, g[1]);
                o.z = sponge_div(o.z, g[2]);
                o.w = sponge_div(o.w, g[3]);
            }
            if (z >= zsmp) {
                const int2 r = sample_plane<MODE>(p, ks, kse, z, tx, ty, o, kpv);
                ks = r.x;
                zsmp = r.y;
            }
            if (colok) {
                const int64_t off = (int64_t)z * p.plane + colo;
                if (CHECK) check_growth(p.status, o);
                *reinterpret_cast<float4 *>(p.u_prev + off) = o;
                if (MODE == kModeStoreD)
                    *reinterpret_cast<ulonglong2 *>(p.dseg_out + off) = make_ulonglong2(dv01, dv23);
                if (MODE == kModeAdjoint) {
                    const float4 dd = ldg4(p.dseg_in + off);
                    float4 ga = *reinterpret_cast<float4 *>(p.gacc + off);
                    ga.x = fmaf(o.x, dd.x, ga.x); ga.y = fmaf(o.y, dd.y, ga.y);
                    ga.z = fmaf(o.z, dd.z, ga.z); ga.w = fmaf(o.w, dd.w, ga.w);
                    *reinterpret_cast<float4 *>(p.gacc + off) = ga;
                }
            }
        }
        if (!ok) break;
    }
    if (!ok) {
        atomicOr(p.status, kStatusTimeout);
        *reinterpret_cast<volatile int *>(&abort_flag) = 1;
    }
}

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
template <int SHAPE, int M, int TY, int MODE>
KernelFn pick_planar_m(bool check)
{
    return check ? step3d_planar<SHAPE, M, MODE, TY, true> : step3d_planar<SHAPE, M, MODE, TY, false>;
}

template <int SHAPE, int M, int TY>
KernelFn pick_planar(int mode, bool check)
{
    if (mode == kModeAdjoint) return pick_planar_m<SHAPE, M, TY, kModeAdjoint>(check);
    if (mode == kModeStoreD) return pick_planar_m<SHAPE, M, TY, kModeStoreD>(check);
    return pick_planar_m<SHAPE, M, TY, kModeForward>(check);
}

template <int M, int TY, int MODE>
KernelFn pick_cross_m(bool check)
{
    return check ? step3d_cross<M, MODE, TY, true> : step3d_cross<M, MODE, TY, false>;
}

template <int M, int TY>
KernelFn pick_cross(int mode, bool check)
{
    if (mode == kModeAdjoint) return pick_cross_m<M, TY, kModeAdjoint>(check);
    if (mode == kModeStoreD) return pick_cross_m<M, TY, kModeStoreD>(check);
    return pick_cross_m<M, TY, kModeForward>(check);
}

KernelFn lookup3(int shape, int M, int ty, int mode, bool check = false)
{
#define FDW_Q(MM, TT) \
    if (shape == FD_CROSS && M == MM && ty == TT) return pick_cross<MM, TT>(mode, check);
    FDW_Q(1, 16) FDW_Q(2, 16) FDW_Q(3, 16) FDW_Q(4, 16) FDW_Q(6, 8) FDW_Q(8, 8)
    FDW_Q(2, 8) FDW_Q(4, 8)
#undef FDW_Q
#define FDW_P(S, MM, TT) \
    if (shape == S && M == MM && ty == TT) return pick_planar<S, MM, TT>(mode, check);
    FDW_P(FD_RHOMBUS, 2, 16) FDW_P(FD_RHOMBUS, 3, 16) FDW_P(FD_RHOMBUS, 4, 16)
    FDW_P(FD_RHOMBUS, 6, 8) FDW_P(FD_RHOMBUS, 8, 8) FDW_P(FD_SQUARE, 2, 16) FDW_P(FD_SQUARE, 4, 16)
    FDW_P(FD_RHOMBUS, 4, 8)
#undef FDW_P
    return nullptr;
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
