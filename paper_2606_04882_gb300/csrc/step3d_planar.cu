// 3D leapfrog step with the rhombus and square stencils (the 2D shape in the
// three coordinate planes), each plane scattered into a register accumulator
// of the outputs it touches.  The kernel lives in its own translation unit so
// that the library builds in parallel; lookup_planar3 returns the
// instantiation for a shape, radius, tile row count, mode and growth check
// (nullptr if none is built).
#include "step3d_common.cuh"

namespace fdw {

namespace {

// ---------------------------------------------------------------------------
// Planar kernel (rhombus, square).
// ---------------------------------------------------------------------------
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

}  // namespace

KernelFn lookup_planar3(int shape, int M, int ty, int mode, bool check)
{
#define FDW_P(S, MM, TT) \
    if (shape == S && M == MM && ty == TT) return pick_planar<S, MM, TT>(mode, check);
    FDW_P(FD_RHOMBUS, 2, 16) FDW_P(FD_RHOMBUS, 3, 16) FDW_P(FD_RHOMBUS, 4, 16)
    FDW_P(FD_RHOMBUS, 6, 8) FDW_P(FD_RHOMBUS, 8, 8) FDW_P(FD_SQUARE, 2, 16) FDW_P(FD_SQUARE, 4, 16)
    FDW_P(FD_RHOMBUS, 4, 8)
#undef FDW_P
    return nullptr;
}

}  // namespace fdw
