// Internal definitions shared by the host runtime (plan.cu) and the kernels.
// Not part of the ABI (see include/fdwave.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/fdwave.h"

namespace fdw {

constexpr int kMaxM = 16;                    // largest radius of any kernel
constexpr int kWDim = kMaxM + 1;             // weight table is W[p][q], p,q in [0, M]
constexpr int kMax3 = 8;                      // largest 3D radius
constexpr int kW3 = kMax3 + 1;
constexpr int kStatusTimeout = 1;            // status word bits
constexpr int kStatusVmax = 2;
constexpr int kStatusBlowup = 4;             // a checked step produced |u| > kBlowupAmp or a non-finite value
constexpr float kBlowupAmp = 1e30f;
constexpr int kCheckEvery = 32;              // steps between growth checks (and the last step)
constexpr long long kWaitCycles = 4000000000LL;   // bound of every device wait (~2 s of SM clocks)

// Point of a per-tile source/receiver table.  Entries of one tile are sorted
// by z.  (x, y) are local to the tile; z is the padded global plane/row.
struct PtEntry {
    int32_t z;
    int32_t yx;      // (y_local << 16) | x_local
    int32_t col;     // column in the series / trace row
    float scale;     // value factor
};

// Launch modes.  The specialised 3D kernels instantiate each mode (the D store
// is compile-time there); the 2D and generic kernels run forward and store-D
// in one instantiation with a run-time branch on dseg_out.  Every mode does the
// same arithmetic, so the checkpointed recompute of the gradient reproduces
// the forward sweep bitwise.
enum Mode : int {
    kModeForward = 0,     // plain step: inject sources, sample receivers
    kModeStoreD = 1,      // forward step that also writes D = kappa * lap to dseg_out
    kModeAdjoint = 2      // adjoint step (q-form) with gradient accumulation
};

// Parameters of one step launch (2D and 3D kernels).
struct StepParams {
    const CUtensorMap *tmap;   // tensor map of the field read by the stencil (halo box)
    const CUtensorMap *tmap_cur_t;    // same field, tile box (no halo)      [3D cross]
    const CUtensorMap *tmap_prev_t;   // u_prev, tile box                     [3D cross]
    const CUtensorMap *tmap_kappa_t;  // kappa, tile box                      [3D cross]
    const float *u_cur;        // the field read by the stencil
    float *u_prev;             // in: older field, out: new field (same buffer)
    const float *kappa;        // (v tau / h)^2 on the padded grid
    int64_t nx, ny, nz;        // padded sizes (ny = 1 in 2D)
    int64_t pitch;             // row pitch in floats
    int64_t plane;             // plane stride in floats (3D)
    int64_t phys_lo[3];        // first physical node per axis (x, y, z) = nb
    int64_t phys_hi[3];        // last physical node per axis (x, y, z)
    float gcoef;               // gamma = gcoef * sum_axes d^2 (d in nodes)
    int tiles_x, tiles_y;      // tiles per axis (3D: x, y; 2D: x, z)
    int zchunk;                // 3D: planes per z-chunk
    int nz_chunks;
    int step;                  // row of the injection series / sample output
    int check;                 // 1: check this step's outputs for growth (kStatusBlowup)
    // bounded waits of the 3D kernels: limit in SM clocks, and (fault-injection
    // test hook, -1 when off) a stream slot whose arrival CTA 0's producer skips
    long long wait_cycles;
    int drop_slot;
    // per-tile point tables (CSR over tiles)
    const int32_t *inj_ptr;
    const PtEntry *inj;
    const float *inj_series;
    int inj_ncol;
    const int32_t *smp_ptr;
    const PtEntry *smp;
    float *smp_out;
    int smp_ncol;
    // FWI
    float *dseg_out;           // kModeStoreD: D written here (same layout as fields)
    const float *dseg_in;      // kModeAdjoint: D^{j-1}
    float *gacc;               // kModeAdjoint: accumulator (same layout as fields)
    int *status;
    float w[kWDim * kWDim];    // symmetric weight table W[p][q] = a_orbit(max, min)
    // 3D kernels (M <= kMax3): the same weights as lane pairs (w, w) for packed
    // FP32x2 arithmetic, W2[p * kW3 + q] = (W[p][q], W[p][q]); and for the
    // planar kernels zp2[i] = (B_i, B_i), zm2[i] = (-B_{i+1}, -B_{i+1}) with
    // B_i = sum_{s >= i} A_s, A_s the total weight of the points at |dz| = s
    // (B_{M+1} = 0)
    unsigned long long w2[kW3 * kW3];
    unsigned long long zp2[kW3 + 1];
    unsigned long long zm2[kW3 + 1];
};

// Batched 2D shots: per-shot descriptor in device memory (128-byte aligned, as
// CUtensorMap is) and the launch parameters of one time step.  ShotInfo is the
// scalar part, which the batched kernel stages into shared memory per tile.
struct ShotInfo {
    float *buf[4];             // buffer 0 holds u^0 at the start, buffer 1 u^{-1};
                               // 2 and 3 are used by the two-step kernel
    const float *kappa;
    const int32_t *inj_ptr;
    const PtEntry *inj;
    const float *inj_series;
    const int32_t *smp_ptr;
    const PtEntry *smp;
    float *smp_out;
    int64_t nx, nz, pitch;
    int64_t phys_lo[3], phys_hi[3];
    float gcoef;
    int tiles_x, inj_ncol, smp_ncol;
    // gradient sweeps of a batch: D of step n of the current segment at
    // dseg + (n - segment start) * field, and the accumulator g
    float *dseg;
    float *gacc;
    int64_t field;             // floats per field buffer
};

struct alignas(128) ShotDesc {
    CUtensorMap tmap[2];       // halo-box maps of field buffers 0 and 1
    CUtensorMap tile[2];       // tile maps (no halo) of field buffers 0 and 1
    CUtensorMap ktile;         // tile map of kappa
    // two-step kernel: u^n box with a 2M-row halo and the u^{n-1} and kappa
    // boxes with an M-row halo, per field buffer (0..3) and for kappa
    CUtensorMap c2[4];
    CUtensorMap p2[4];
    CUtensorMap k2;
    ShotInfo info;
};

// One tile of a batch: its shot, its index and origin in the shot's grid, and
// its ranges in the shot's injection and sampling tables.
struct alignas(16) TileRec {
    int shot, tile, x0, z0, ib, ie, sb, se;
    int xb, xe;                // two-step kernel: range in BatchParams::ext
    int pad[2];
};

struct BatchParams {
    const ShotDesc *shots;
    const TileRec *tiles;      // every shot's tiles, shot by shot
    // two-step kernel: source entries of each tile's extended region (x
    // relative to the region's origin), and the buffers holding u^n, u^{n-1}
    // and receiving u^{n+1}, u^{n+2}
    const PtEntry *ext;
    int roles[4];
    int ntiles;                // tiles of all shots
    int step;                  // time step n (series row)
    int parity;                // field buffer (0 or 1 of the descriptor) holding the stencil input
    int seg;                   // gradient sweeps: index of this step's D in its segment
    int check;                 // 1: check this step's outputs for growth (kStatusBlowup)
    int *status;
    float w[kWDim * kWDim];
};

// Persistent 2D time loop: step parameters plus both buffers' maps and the
// grid-barrier words (in the workspace's status block).
struct PersistParams {
    StepParams base;
    const CUtensorMap *maps;   // halo-box map of buffer b at maps[2 b] (workspace map layout)
    float *buf[2];
    int nt;
    unsigned int *bar_count;
    unsigned int *bar_gen;
    int *abort_flag;
};

// Kernel variant descriptor chosen by the plan.
struct Variant {
    int dim, shape, M, N;
    int generic;       // 1: runtime-M kernel
    int tx, tz;        // 2D tile: columns, rows of output per CTA; 3D: x, y
    int threads;
    size_t smem;
    int box[3];        // TMA box with halo (x, y, z)
    int tbox[2];       // TMA tile box without halo (x, y) [3D cross]
};

// Host launchers (defined in the .cu files).
int select_variant_2d(int shape, int M, int N, int64_t nx, int64_t nz, Variant *v, int r_pref = 0);
int select_variant_3d(int shape, int M, int N, int64_t nx, int64_t ny, int64_t nz, Variant *v,
                      int ty_pref = 0);
// Tuning candidates: rows per thread (2D) / y tile (3D) with a kernel.
int variants_2d(int shape, int M, int *r_out, int cap);
int variants_3d(int shape, int M, int *ty_out, int cap);
constexpr int kMaxVariants = 8;

cudaError_t launch_step2d(const Variant &v, int mode, const StepParams &p, cudaStream_t s);
cudaError_t launch_step3d(const Variant &v, int mode, const StepParams &p, cudaStream_t s);
int occupancy_3d(const Variant &v);
// Every step of a single-launch batch in one cooperative launch (grid barrier
// between steps; the status block of bp.status holds its words).
cudaError_t launch_batched2d_persistent(const Variant &v, const BatchParams &bp, int ntiles, int nt,
                                       cudaStream_t s);
int batch2d_variant(int shape, int M, int64_t total_tiles4, Variant *v, int r_pref = 0);
int batch2d_variants(int shape, int M, int *r_out, int cap);
int persist2d_grid(const Variant &v, int ntiles);
cudaError_t launch_persist2d(const Variant &v, const PersistParams &pp, int grid, cudaStream_t s);
cudaError_t launch_batched2d(const Variant &v, const BatchParams &bp, int ntiles, cudaStream_t s,
                             int mode = kModeForward);
// Two-step batched kernel (u^{n+1} and u^{n+2} per pass): geometry of its
// boxes for cross stencils with M <= 4 (FD_ERR_UNSUPPORTED otherwise).
struct Batch2Geo {
    int tz, hx, hxc;           // tile rows; x halo of the extended region; x halo of the u^n box
    int cbox[2], pbox[2];      // u^n box and u^{n-1} / kappa box (x, z extents)
};
int batch2d2_geometry(int shape, int M, Batch2Geo *g);
cudaError_t launch_batched2d2(const Variant &v, const BatchParams &bp, int ntiles, cudaStream_t s);

// aux kernels
cudaError_t launch_prep_kappa(const float *model, int kind, float *kappa, int dim,
                              const int64_t phys[3], int nb, const int64_t pad[3],
                              int64_t pitch, int64_t plane, double dt_over_h,
                              float vmax_sq_limit, int *status, cudaStream_t s);
cudaError_t launch_copy_state(const float *src, int64_t src_pitch, int64_t src_plane,
                              float *dst, int64_t dst_pitch, int64_t dst_plane,
                              const int64_t pad[3], cudaStream_t s);
cudaError_t launch_fold_grad(const float *gacc, int64_t pitch, int64_t plane,
                             const int64_t phys[3], int nb, float scale, float *grad,
                             cudaStream_t s);

// Driver entry point for cuTensorMapEncodeTiled (resolved at run time).
int encode_tmap(CUtensorMap *map, const float *base, int rank, const int64_t *dims,
                const int64_t *strides_bytes, const int *box);

}  // namespace fdw
