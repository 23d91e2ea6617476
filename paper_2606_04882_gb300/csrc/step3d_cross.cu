// 3D leapfrog step with the cross stencil (the 3D cross of Eq.
// spacexz_derivative2_sym: six axis arms), z arm in a register queue.  The
// kernel lives in its own translation unit so that the library builds in
// parallel; lookup_cross3 returns the instantiation for a radius, tile row
// count, mode and growth check (nullptr if none is built).
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

}  // namespace

KernelFn lookup_cross3(int M, int ty, int mode, bool check)
{
#define FDW_Q(MM, TT) \
    if (M == MM && ty == TT) return pick_cross<MM, TT>(mode, check);
    FDW_Q(1, 16) FDW_Q(2, 16) FDW_Q(3, 16) FDW_Q(4, 16) FDW_Q(6, 8) FDW_Q(8, 8)
    FDW_Q(2, 8) FDW_Q(4, 8)
#undef FDW_Q
    return nullptr;
}

}  // namespace fdw
