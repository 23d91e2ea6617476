// Host runtime of libfdwave: plans, workspace layout, point tables, the
// forward time loop, the checkpointed adjoint gradient and batched shots.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "internal.h"
#include "runtime.h"

struct fd_plan {
    fd_problem prob;
    fd_stencil_desc st;
    std::vector<std::array<int, 3>> keys;
    std::vector<int> mult;
    std::vector<double> w;
    double cmax = 0.0;
    int shape_eff = 0;
    int64_t pad[3] = {1, 1, 1};   // (z, y, x)
    int64_t pitch = 0, plane = 0, field = 0;   // floats
    fdw::Variant var{};
    int tiles_x = 0, tiles_y = 0, ntiles = 0;
    int max_tiles = 0;   // largest tile count of any variant the plan can take
    int zchunk = 0, nz_chunks = 1;
    bool tuned = false;
    float gcoef = 0.f;
    float W[fdw::kWDim * fdw::kWDim];
    void *last_ws = nullptr;
    // (workspace, hash of the source and receiver indices) of the recent
    // fd_gradient_forward calls, newest last: the states fd_gradient_adjoint
    // accepts (cleared when the kernel variant changes)
    std::vector<std::pair<void *, uint64_t>> stores;
    uint64_t id = 0;   // unique per created plan (never reused: keys the graph cache)
};

// FNV-1a over the source and receiver counts and indices (host arrays): the
// identity of a stored forward's point tables
static uint64_t points_hash(int nsrc, const int64_t *src, int nrec, const int64_t *rec)
{
    uint64_t h = 1469598103934665603ull;
    auto mix = [&h](uint64_t v) {
        for (int b = 0; b < 8; ++b) {
            h ^= (v >> (8 * b)) & 0xffu;
            h *= 1099511628211ull;
        }
    };
    mix((uint64_t)nsrc);
    for (int i = 0; i < nsrc && src; ++i) mix((uint64_t)src[i]);
    mix((uint64_t)nrec);
    for (int i = 0; i < nrec && rec; ++i) mix((uint64_t)rec[i]);
    return h;
}

// Forget a workspace as a stored forward (another call is about to write it)
static void forget_store(fd_plan *p, void *ws)
{
    for (size_t i = 0; i < p->stores.size(); ++i)
        if (p->stores[i].first == ws) {
            p->stores.erase(p->stores.begin() + (long)i);
            return;
        }
}

namespace fdw {

// Set while fd_plan_autotune times candidates: their time loops are captured
// into graphs kept here instead of the shared cache (so that no candidate
// evicts a caller's graph), and destroyed when tuning ends.
thread_local std::map<std::vector<uint64_t>, cudaGraphExec_t> *t_tune_graphs = nullptr;

namespace {

thread_local char g_err[512] = "";

constexpr size_t kAlign = 256;
inline size_t up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }

#define FDW_CK(call)                                                                     \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return set_error(FD_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

int set_error(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

void clear_error() { g_err[0] = 0; }

namespace {

// ----------------------------- workspace layout ---------------------------

struct Layout {
    size_t status = 0, tmaps = 0, kappa = 0, buf[4] = {0, 0, 0, 0}, gacc = 0, ckpt = 0, dseg = 0;
    size_t tab = 0, tab_bytes = 0;
    size_t total = 0;
    int n_tmaps = 2, nck = 0, kseg = 0;
};

struct Tables {
    std::vector<char> blob;           // host image of the table region
    size_t inj_ptr = 0, inj = 0, smp_ptr = 0, smp = 0;   // offsets inside blob
    size_t ainj_ptr = 0, ainj = 0, asmp_ptr = 0, asmp = 0;
    bool has_adj = false;
};

// Tile geometry the point tables are built for.
struct TileGeo {
    int tx, tz, tiles_x, ntiles;
};

TileGeo plan_geo(const fd_plan *p) { return {p->var.tx, p->var.tz, p->tiles_x, p->ntiles}; }

size_t table_bytes_n(int ntiles, int nsrc, int nrec, bool adj)
{
    const size_t ptr = up((ntiles + 1) * sizeof(int32_t));
    size_t b = 2 * ptr + up(std::max(nsrc, 1) * sizeof(PtEntry)) + up(std::max(nrec, 1) * sizeof(PtEntry));
    return adj ? 2 * b : b;
}

// Point tables are sized for the plan's largest tile count, so that one
// workspace size serves every kernel variant (the default, each autotune
// candidate and the tuned choice).
size_t table_bytes(const fd_plan *p, int nsrc, int nrec, bool adj)
{
    return table_bytes_n(std::max(p->ntiles, p->max_tiles), nsrc, nrec, adj);
}

Layout make_layout(const fd_plan *p, int nsrc, int nrec, bool grad, int kseg, int ntiles_tab = -1)
{
    Layout L;
    const size_t fb = up(p->field * sizeof(float));
    size_t o = 0;
    L.status = o; o += kAlign;
    L.n_tmaps = 2 * (grad ? 4 : 2) + 1;   // (halo box, tile box) per buffer + kappa tile box
    L.tmaps = o; o += up(L.n_tmaps * sizeof(CUtensorMap));
    L.kappa = o; o += fb;
    for (int i = 0; i < (grad ? 4 : 2); ++i) { L.buf[i] = o; o += fb; }
    if (grad) {
        L.gacc = o; o += fb;
        L.kseg = kseg;
        L.nck = (p->prob.nt + kseg - 1) / kseg;
        L.ckpt = o; o += (size_t)2 * L.nck * fb;
        L.dseg = o; o += (size_t)kseg * fb;
    }
    L.tab = o;
    L.tab_bytes = ntiles_tab >= 0 ? table_bytes_n(ntiles_tab, nsrc, nrec, grad)
                                  : table_bytes(p, nsrc, nrec, grad);
    o += L.tab_bytes;
    L.total = o;
    return L;
}

// Map physical linear indices to tile tables (CSR over tiles, z-sorted).
struct Pt {
    int tile;
    PtEntry e;
};

int locate(const fd_plan *p, const TileGeo &G, int64_t idx, int col, float scale, Pt &out)
{
    const fd_problem &pr = p->prob;
    const int64_t nphys = pr.n[0] * pr.n[1] * pr.n[2];
    if (idx < 0 || idx >= nphys) return set_error(FD_ERR_ARG, "point index %lld outside the physical grid", (long long)idx);
    const int64_t ix = idx % pr.n[2], r = idx / pr.n[2], iy = r % pr.n[1], iz = r / pr.n[1];
    const int64_t x = ix + pr.nb, z = iz + pr.nb, y = pr.dim == 3 ? iy + pr.nb : 0;
    const int tx = (int)(x / G.tx);
    int tile;
    int64_t yl;
    if (pr.dim == 2) {
        tile = (int)(z / G.tz) * G.tiles_x + tx;
        yl = 0;
    } else {
        tile = (int)(y / G.tz) * G.tiles_x + tx;
        yl = y % G.tz;
    }
    out.tile = tile;
    out.e.z = (int32_t)z;
    out.e.yx = (int32_t)((yl << 16) | (x % G.tx));
    out.e.col = col;
    out.e.scale = scale;
    return FD_OK;
}

int build_table(const fd_plan *p, const TileGeo &G, int n, const int64_t *idx, float scale,
                std::vector<int32_t> &ptr, std::vector<PtEntry> &ent)
{
    std::vector<Pt> pts(n);
    for (int i = 0; i < n; ++i) {
        int st = locate(p, G, idx[i], i, scale, pts[i]);
        if (st) return st;
    }
    // by tile, then z, then (y, x): the kernels find a plane's and a thread's
    // entries by binary search
    std::stable_sort(pts.begin(), pts.end(), [](const Pt &a, const Pt &b) {
        if (a.tile != b.tile) return a.tile < b.tile;
        if (a.e.z != b.e.z) return a.e.z < b.e.z;
        return (uint32_t)a.e.yx < (uint32_t)b.e.yx;
    });
    ptr.assign(G.ntiles + 1, 0);
    for (auto &q : pts) ptr[q.tile + 1]++;
    for (int t = 0; t < G.ntiles; ++t) ptr[t + 1] += ptr[t];
    ent.resize(pts.size());
    for (size_t i = 0; i < pts.size(); ++i) ent[i] = pts[i].e;
    return FD_OK;
}

int make_tables(const fd_plan *p, int nsrc, const int64_t *src, int nrec, const int64_t *rec,
                bool adj, Tables &T, const TileGeo *geo = nullptr)
{
    const TileGeo G = geo ? *geo : plan_geo(p);
    const fd_problem &pr = p->prob;
    const double hd = std::pow(pr.h, pr.dim);
    const float src_scale = (float)(pr.dt * pr.dt / hd);
    std::vector<int32_t> a, b, c, d;
    std::vector<PtEntry> ea, eb, ec, ed;
    int st;
    if ((st = build_table(p, G, nsrc, src, src_scale, a, ea))) return st;
    if ((st = build_table(p, G, nrec, rec, 1.0f, b, eb))) return st;
    if (adj) {
        // adjoint (q = s2 nu form): residual injected as kappa * h^2 * r (kappa applied
        // in the kernel); source samples give dJ/ds = q tau^2 / (h^dim h^2 kappa)
        if ((st = build_table(p, G, nrec, rec, (float)(pr.h * pr.h), c, ec))) return st;
        if ((st = build_table(p, G, nsrc, src, (float)(pr.dt * pr.dt / (hd * pr.h * pr.h)), d, ed))) return st;
    }
    const size_t ptrb = up((G.ntiles + 1) * sizeof(int32_t));
    const size_t sb = up(std::max(nsrc, 1) * sizeof(PtEntry)), rb = up(std::max(nrec, 1) * sizeof(PtEntry));
    T.blob.assign(table_bytes_n(G.ntiles, nsrc, nrec, adj), 0);
    size_t o = 0;
    auto put = [&](size_t &off, const void *src_, size_t bytes, size_t span) {
        off = o;
        if (bytes) std::memcpy(T.blob.data() + o, src_, bytes);
        o += span;
    };
    put(T.inj_ptr, a.data(), a.size() * 4, ptrb);
    put(T.inj, ea.data(), ea.size() * sizeof(PtEntry), sb);
    put(T.smp_ptr, b.data(), b.size() * 4, ptrb);
    put(T.smp, eb.data(), eb.size() * sizeof(PtEntry), rb);
    T.has_adj = adj;
    if (adj) {
        put(T.ainj_ptr, c.data(), c.size() * 4, ptrb);
        put(T.ainj, ec.data(), ec.size() * sizeof(PtEntry), rb);
        put(T.asmp_ptr, d.data(), d.size() * 4, ptrb);
        put(T.asmp, ed.data(), ed.size() * sizeof(PtEntry), sb);
    }
    return FD_OK;
}

// ------------------------------- tuning -----------------------------------

int ensure_tuned(fd_plan *p)
{
    if (p->tuned) return FD_OK;
    if (p->prob.dim == 3) {
        int dev = 0, nsm = 152, occ = 1;
        FDW_CK(cudaGetDevice(&dev));
        FDW_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        occ = std::max(1, occupancy_3d(p->var));
        const int64_t slots = (int64_t)nsm * occ;
        const int M = p->st.M;
        double best = 1e300;
        int bestc = 1;
        for (int c = 1; c <= 64; ++c) {
            const int64_t chunk = (p->pad[0] + c - 1) / c;
            if (c > 1 && chunk < 2 * M) break;
            const int64_t ctas = (int64_t)p->ntiles * c;
            const double waves = std::ceil((double)ctas / slots);
            const double cost = waves * (chunk + 0.5 * 2 * M);
            if (cost < best * 0.999) { best = cost; bestc = c; }
        }
        p->zchunk = (int)((p->pad[0] + bestc - 1) / bestc);
        p->nz_chunks = (int)((p->pad[0] + p->zchunk - 1) / p->zchunk);
    }
    p->tuned = true;
    return FD_OK;
}

void fill_params(const fd_plan *p, StepParams &sp)
{
    std::memset(&sp, 0, sizeof sp);
    sp.nz = p->pad[0];
    sp.ny = p->pad[1];
    sp.nx = p->pad[2];
    sp.pitch = p->pitch;
    sp.plane = p->plane;
    const fd_problem &pr = p->prob;
    sp.phys_lo[0] = pr.nb; sp.phys_hi[0] = pr.nb + pr.n[2] - 1;
    if (pr.dim == 3) { sp.phys_lo[1] = pr.nb; sp.phys_hi[1] = pr.nb + pr.n[1] - 1; }
    sp.phys_lo[2] = pr.nb; sp.phys_hi[2] = pr.nb + pr.n[0] - 1;
    sp.gcoef = p->gcoef;
    sp.tiles_x = p->tiles_x;
    sp.tiles_y = p->tiles_y;
    sp.zchunk = p->zchunk;
    sp.nz_chunks = p->nz_chunks;
    sp.wait_cycles = kWaitCycles;
    sp.drop_slot = -1;
    std::memcpy(sp.w, p->W, sizeof sp.w);
    // packed 3D weight tables, from the FP32 table
    auto pair = [](float v) {
        uint32_t b;
        std::memcpy(&b, &v, 4);
        return ((unsigned long long)b << 32) | b;
    };
    for (int a = 0; a < kW3; ++a)
        for (int c = 0; c < kW3; ++c) sp.w2[a * kW3 + c] = pair(p->W[a * kWDim + c]);
    const int M = p->st.M;
    double A[kW3 + 1] = {0.0};
    for (int s = 1; s <= M && s < kW3; ++s) {
        const int E = shape_ext(p->shape_eff, M, 0, s);
        double a = p->W[s];
        for (int pp = 1; pp <= E; ++pp) a += 4.0 * p->W[pp * kWDim + s];
        A[s] = a;
    }
    double B = 0.0;
    for (int i = std::min(M, kW3 - 1); i >= 1; --i) {
        B += A[i];
        sp.zp2[i] = pair((float)B);
        sp.zm2[i - 1] = pair(-(float)B);
    }
}

cudaError_t launch(const fd_plan *p, int mode, const StepParams &sp, cudaStream_t s)
{
    return p->prob.dim == 2 ? launch_step2d(p->var, mode, sp, s) : launch_step3d(p->var, mode, sp, s);
}

// Tensor map of one field buffer: halo box (tile = false) or tile box.
int encode_field_map(const fd_plan *p, CUtensorMap *map, const float *base, bool tile)
{
    int64_t dims[3], str[2];
    int box[3];
    if (p->prob.dim == 2) {
        dims[0] = p->pad[2]; dims[1] = p->pad[0];
        str[0] = p->pitch * 4;
        box[0] = tile ? p->var.tbox[0] : p->var.box[0];
        box[1] = tile ? p->var.tbox[1] : p->var.box[1];
        return encode_tmap(map, base, 2, dims, str, box);
    }
    dims[0] = p->pad[2]; dims[1] = p->pad[1]; dims[2] = p->pad[0];
    str[0] = p->pitch * 4; str[1] = p->plane * 4;
    if (tile) {
        box[0] = p->var.tbox[0]; box[1] = p->var.tbox[1];
    } else {
        box[0] = p->var.box[0]; box[1] = p->var.box[1];
    }
    box[2] = 1;
    return encode_tmap(map, base, 3, dims, str, box);
}

// Point the step parameters at buffer `cur` (stencil input) and `prev` (u_prev).
void bind_maps(StepParams &sp, const CUtensorMap *maps, int nbuf, int cur, int prev)
{
    sp.tmap = maps + 2 * cur;
    sp.tmap_cur_t = maps + 2 * cur + 1;
    sp.tmap_prev_t = maps + 2 * prev + 1;
    sp.tmap_kappa_t = maps + 2 * nbuf;
}

// Growth check on every kCheckEvery-th step and on the last one.
inline int check_step(int n, int nt) { return (n + 1) % kCheckEvery == 0 || n + 1 == nt; }

// Fault-injection test hook that faults nothing.  FDWAVE_DEBUG_WAIT_CYCLES=<c>
// bounds every wait of the 3D kernels by c SM clocks, and
// FDWAVE_DEBUG_DROP_SLOT=<s> makes the producer of CTA 0 skip stream slot s:
// that CTA's consumers then wait for copies that never come, give up after c
// clocks and report FD_ERR_TIMEOUT through the status word, and the producer
// gives up on their release the same way.  A call with the hook set launches
// its steps one by one (no graph is captured or replayed).  Returns true when
// the hook is set.
bool debug_hook(const fd_plan *p, StepParams &sp)
{
    if (p->prob.dim != 3) return false;
    const char *c = getenv("FDWAVE_DEBUG_WAIT_CYCLES");
    const char *d = getenv("FDWAVE_DEBUG_DROP_SLOT");
    bool on = false;
    if (c && *c) {
        const long long v = atoll(c);
        if (v > 0) { sp.wait_cycles = v; on = true; }
    }
    if (d && *d) {
        sp.drop_slot = atoi(d);
        on = true;
    }
    return on;
}

int check_common(const fd_plan *p, int model_kind, const float *model, int nsrc,
                 const int64_t *src, const float *wav, int nrec, const int64_t *rec, void *ws,
                 size_t ws_bytes, size_t need)
{
    if (!p) return set_error(FD_ERR_ARG, "plan is NULL");
    if (model_kind != FD_MODEL_VELOCITY && model_kind != FD_MODEL_SLOWNESS2)
        return set_error(FD_ERR_ARG, "unknown model kind %d", model_kind);
    if (!model) return set_error(FD_ERR_ARG, "model is NULL");
    if (nsrc < 0 || nrec < 0) return set_error(FD_ERR_ARG, "negative source/receiver count");
    if (nsrc > 0 && (!src || !wav)) return set_error(FD_ERR_ARG, "sources need indices and a wavelet");
    if (nrec > 0 && !rec) return set_error(FD_ERR_ARG, "receivers need indices");
    if (!ws) return set_error(FD_ERR_ARG, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return set_error(FD_ERR_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < need)
        return set_error(FD_ERR_NOMEM, "workspace has %zu bytes, needs %zu", ws_bytes, need);
    return FD_OK;
}

}  // namespace
}  // namespace fdw

using namespace fdw;

// --------------------------------- ABI ------------------------------------

extern "C" const char *fd_last_error(void) { return g_err; }

extern "C" const char *fd_version(void) { return "fdwave 0.1 (sm_103a)"; }

extern "C" int fd_plan_create(const fd_problem *prob, const fd_stencil_desc *stencil, fd_plan **out)
{
    clear_error();
    if (!prob || !stencil || !out) return set_error(FD_ERR_ARG, "NULL argument to fd_plan_create");
    *out = nullptr;
    const fd_problem &pr = *prob;
    if (pr.dim != 2 && pr.dim != 3) return set_error(FD_ERR_ARG, "dim must be 2 or 3");
    if (stencil->dim != pr.dim) return set_error(FD_ERR_ARG, "stencil dim %d != problem dim %d", stencil->dim, pr.dim);
    if (pr.n[0] < 1 || pr.n[2] < 1 || pr.n[1] < 1 || (pr.dim == 2 && pr.n[1] != 1))
        return set_error(FD_ERR_ARG, "grid sizes must be >= 1 (ny = 1 in 2D)");
    if (pr.nb < 0 || pr.nt < 0) return set_error(FD_ERR_ARG, "nb and nt must be >= 0");
    if (!(pr.h > 0) || !(pr.dt > 0) || !(pr.vmax > 0)) return set_error(FD_ERR_ARG, "h, dt and vmax must be > 0");
    const int64_t padx = pr.n[2] + 2 * pr.nb, pady = pr.dim == 3 ? pr.n[1] + 2 * pr.nb : 1,
                  padz = pr.n[0] + 2 * pr.nb;
    if (padx > (1 << 24) || pady > (1 << 24) || padz > (1 << 24) || padx * pady * padz > (int64_t)1 << 36)
        return set_error(FD_ERR_ARG, "grid too large");
    if (padx >= 65536 * 64 || (pr.dim == 3 && pady > 32767 * 16))
        return set_error(FD_ERR_ARG, "grid too large for the tile tables");
    fd_plan *p = new (std::nothrow) fd_plan();
    if (!p) return set_error(FD_ERR_NOMEM, "host allocation failed");
    static std::atomic<uint64_t> next_id{1};
    p->id = next_id.fetch_add(1);
    p->prob = pr;
    p->st = *stencil;
    int st = compute_weights(stencil, p->keys, p->mult, p->w, nullptr, nullptr);
    if (!st) st = compute_cfl(stencil, p->w, &p->cmax);
    if (st) { delete p; return st; }
    const double C = pr.vmax * pr.dt / pr.h;
    if (C > p->cmax * (1.0 + 1e-12)) {
        const double cmax = p->cmax;
        delete p;
        return set_error(FD_ERR_UNSTABLE, "Courant number %.6g exceeds the stability limit %.6g", C, cmax);
    }
    // weight table W[p][q] and the effective shape (all-zero off-axis orbits -> cross)
    std::memset(p->W, 0, sizeof p->W);
    bool offaxis = false;
    for (size_t k = 0; k < p->keys.size(); ++k) {
        const int a = p->keys[k][0], b = p->keys[k][1];
        const float v = (float)p->w[k];
        p->W[a * kWDim + b] = v;
        p->W[b * kWDim + a] = v;
        if (b != 0 && p->w[k] != 0.0) offaxis = true;
    }
    p->shape_eff = offaxis ? stencil->shape : FD_CROSS;
    p->pad[0] = padz; p->pad[1] = pady; p->pad[2] = padx;
    p->pitch = (padx + 31) / 32 * 32;
    p->plane = pr.dim == 3 ? p->pitch * pady : p->pitch * padz;
    p->field = pr.dim == 3 ? p->plane * padz : p->plane;
    p->field = (p->field + 63) / 64 * 64;
    const int M = stencil->M;
    if (pr.dim == 2) {
        st = select_variant_2d(p->shape_eff, M, stencil->N, padx, padz, &p->var);
        p->tiles_x = (int)((padx + p->var.tx - 1) / p->var.tx);
        p->tiles_y = (int)((padz + p->var.tz - 1) / p->var.tz);
    } else {
        st = select_variant_3d(p->shape_eff, M, stencil->N, padx, pady, padz, &p->var);
        p->tiles_x = (int)((padx + p->var.tx - 1) / p->var.tx);
        p->tiles_y = (int)((pady + p->var.tz - 1) / p->var.tz);
        p->zchunk = (int)padz;
        p->nz_chunks = 1;
    }
    if (st) {
        const int shape_eff = p->shape_eff;
        delete p;
        return set_error(FD_ERR_UNSUPPORTED, "no kernel for shape %d, M %d in %dD", shape_eff, M, pr.dim);
    }
    p->ntiles = p->tiles_x * p->tiles_y;
    p->max_tiles = p->ntiles;
    {
        int prefs[kMaxVariants];
        const int np = pr.dim == 2 ? variants_2d(p->shape_eff, M, prefs, kMaxVariants)
                                   : variants_3d(p->shape_eff, M, prefs, kMaxVariants);
        for (int i = 0; i < np; ++i) {
            Variant v;
            if (pr.dim == 2 ? select_variant_2d(p->shape_eff, M, stencil->N, padx, padz, &v, prefs[i])
                            : select_variant_3d(p->shape_eff, M, stencil->N, padx, pady, padz, &v, prefs[i]))
                continue;
            const int64_t n = ((padx + v.tx - 1) / v.tx) *
                              (((pr.dim == 2 ? padz : pady) + v.tz - 1) / v.tz);
            p->max_tiles = (int)std::max<int64_t>(p->max_tiles, n);
        }
    }
    if (pr.nb > 0) {
        const double R = pr.damp_R > 0 ? pr.damp_R : 1e-3;
        const double eta_max = 3.0 * pr.vmax * std::log(1.0 / R) / (2.0 * pr.nb * pr.h);
        p->gcoef = (float)(0.5 * pr.dt * eta_max / ((double)pr.nb * pr.nb));
    }
    *out = p;
    return FD_OK;
}

extern "C" void fd_plan_destroy(fd_plan *plan) { delete plan; }

// ------------------------------- autotuner --------------------------------
namespace {

// Re-derive the tile counts of a plan for a kernel variant.
void apply_variant(fd_plan *p, const Variant &v)
{
    p->var = v;
    p->tiles_x = (int)((p->pad[2] + v.tx - 1) / v.tx);
    p->tiles_y = (int)(((p->prob.dim == 2 ? p->pad[0] : p->pad[1]) + v.tz - 1) / v.tz);
    p->ntiles = p->tiles_x * p->tiles_y;
    p->tuned = false;
}

struct TuneChoice {
    int pref;        // rows per thread (2D) or y tile (3D)
    int zchunk;      // 3D z-chunk (0 in 2D)
};

std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune;

std::string tune_key(const fd_plan *p)
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, dev);
    char buf[256];
    snprintf(buf, sizeof buf, "%s|%d|%d|%d|%d|%lld|%lld|%lld", prop.name, p->prob.dim, p->shape_eff,
             p->st.M, p->st.N, (long long)p->pad[0], (long long)p->pad[1], (long long)p->pad[2]);
    for (char *c = buf; *c; ++c)
        if (*c == ' ') *c = '_';
    return buf;
}

void tune_file_load()
{
    static bool done = false;
    const char *path = getenv("FDWAVE_TUNE_CACHE");
    if (done || !path) return;
    done = true;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char key[256];
    int a, b;
    while (fscanf(f, "%255s %d %d", key, &a, &b) == 3) g_tune[key] = {a, b};
    fclose(f);
}

void tune_file_store(const std::string &key, const TuneChoice &c)
{
    const char *path = getenv("FDWAVE_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d\n", key.c_str(), c.pref, c.zchunk);
    fclose(f);
}

int apply_choice(fd_plan *p, const TuneChoice &c)
{
    Variant v;
    const int M = p->st.M;
    int st = p->prob.dim == 2
                 ? select_variant_2d(p->shape_eff, M, p->st.N, p->pad[2], p->pad[0], &v, c.pref)
                 : select_variant_3d(p->shape_eff, M, p->st.N, p->pad[2], p->pad[1], p->pad[0], &v, c.pref);
    if (st) return st;
    apply_variant(p, v);
    if (p->prob.dim == 3) {
        p->zchunk = c.zchunk;
        p->nz_chunks = (int)((p->pad[0] + c.zchunk - 1) / c.zchunk);
        p->tuned = true;
    } else {
        p->tuned = true;
    }
    return FD_OK;
}

}  // namespace

extern "C" int fd_plan_autotune(fd_plan *p, int model_kind, const float *model, void *ws,
                                size_t ws_bytes, void *stream)
{
    clear_error();
    if (!p) return set_error(FD_ERR_ARG, "plan is NULL");
    p->stores.clear();   // a stored forward's tables belong to the old variant
    size_t need = make_layout(p, 0, 0, false, 1).total;
    // variants with more tiles need larger tables: size for the worst case
    need += 4 * kAlign;
    int st = check_common(p, model_kind, model, 0, nullptr, nullptr, 0, nullptr, ws, ws_bytes, 0);
    if (st) return st;
    if (ws_bytes < need) return set_error(FD_ERR_NOMEM, "autotune workspace has %zu bytes, needs %zu", ws_bytes, need);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_file_load();
    const std::string key = tune_key(p);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return apply_choice(p, it->second);
    if (p->var.generic) return FD_OK;   // a single kernel: nothing to choose
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int prefs[kMaxVariants];
    const int np = p->prob.dim == 2 ? variants_2d(p->shape_eff, p->st.M, prefs, kMaxVariants)
                                    : variants_3d(p->shape_eff, p->st.M, prefs, kMaxVariants);
    std::vector<TuneChoice> cands;
    for (int i = 0; i < np; ++i) {
        if (p->prob.dim == 2) {
            cands.push_back({prefs[i], 0});
            continue;
        }
        fd_plan q = *p;
        if (apply_choice(&q, {prefs[i], (int)q.pad[0]})) continue;
        q.tuned = false;
        if ((st = ensure_tuned(&q))) return st;        // cost-model z-chunk for this tile
        const int base = q.zchunk;
        for (int f : {1, 2, 4}) {
            const int zc = std::max(2 * p->st.M, base / f);
            if (f > 1 && zc == cands.back().zchunk) continue;
            cands.push_back({prefs[i], zc});
        }
        if (base * 2 <= q.pad[0]) cands.push_back({prefs[i], base * 2});
    }
    if (cands.empty()) return set_error(FD_ERR_UNSUPPORTED, "no kernel variant to tune");
    cudaEvent_t e0, e1;
    FDW_CK(cudaEventCreate(&e0));
    FDW_CK(cudaEventCreate(&e1));
    float best = 1e30f;
    TuneChoice bestc = cands[0];
    // Time per step of a candidate: (best of three 64-step runs - best of three
    // 16-step runs) / 48, both run as captured graphs like a caller's long
    // runs, which leaves out the set-up of each call (kappa, tables) and the
    // first steps' ramp.
    struct Tuning {
        std::map<std::vector<uint64_t>, cudaGraphExec_t> graphs;
        cudaStream_t s;
        explicit Tuning(cudaStream_t st) : s(st) { t_tune_graphs = &graphs; }
        ~Tuning()
        {
            t_tune_graphs = nullptr;
            cudaStreamSynchronize(s);
            for (auto &g : graphs) cudaGraphExecDestroy(g.second);
        }
    } tuning(s);
    auto timed = [&](fd_plan &q, int nt, float &out) -> int {
        q.prob.nt = nt;
        out = 1e30f;
        for (int r = 0; r < 3; ++r) {
            FDW_CK(cudaEventRecord(e0, s));
            const int rs = fd_forward(&q, model_kind, model, 0, nullptr, nullptr, 0, nullptr, nullptr,
                                      nullptr, nullptr, ws, ws_bytes, stream);
            if (rs) return rs;
            FDW_CK(cudaEventRecord(e1, s));
            FDW_CK(cudaEventSynchronize(e1));
            float t = 0.f;
            FDW_CK(cudaEventElapsedTime(&t, e0, e1));
            out = std::min(out, t);
        }
        return FD_OK;
    };
    for (const TuneChoice &c : cands) {
        fd_plan q = *p;
        if (apply_choice(&q, c)) continue;
        q.prob.nt = 64;
        if (make_layout(&q, 0, 0, false, 1).total > ws_bytes) continue;
        st = fd_forward(&q, model_kind, model, 0, nullptr, nullptr, 0, nullptr, nullptr, nullptr,
                        nullptr, ws, ws_bytes, stream);     // warm-up
        if (st) break;
        float t64 = 0.f, t16 = 0.f;
        if ((st = timed(q, 64, t64)) || (st = timed(q, 16, t16))) break;
        const float ms = (t64 - t16) / 48.f;
        if (const char *vb = getenv("FDWAVE_TUNE_VERBOSE"))
            if (vb[0] == '1')
                fprintf(stderr, "fdwave tune %s: tile %d z-chunk %d: %.4f ms per step\n",
                        key.c_str(), c.pref, c.zchunk, ms);
        // a later candidate must win by 2 %: the first of each tile shape is
        // the cost model's z-chunk, and near-ties are timing noise
        if (ms < 0.98f * best) {
            best = ms;
            bestc = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    g_tune[key] = bestc;
    tune_file_store(key, bestc);
    return apply_choice(p, bestc);
}

extern "C" int fd_plan_variants(const fd_plan *p, int cap, int *n, int *variants)
{
    clear_error();
    if (!p || !n || cap < 0 || (cap > 0 && !variants)) return set_error(FD_ERR_ARG, "bad argument");
    int prefs[kMaxVariants];
    const int np = p->var.generic ? 0
                 : p->prob.dim == 2 ? variants_2d(p->shape_eff, p->st.M, prefs, kMaxVariants)
                                    : variants_3d(p->shape_eff, p->st.M, prefs, kMaxVariants);
    *n = np;
    for (int i = 0; i < np && i < cap; ++i) variants[i] = prefs[i];
    return FD_OK;
}

extern "C" int fd_plan_set_variant(fd_plan *p, int variant, int z_chunk)
{
    clear_error();
    if (!p || z_chunk < 0) return set_error(FD_ERR_ARG, "bad argument");
    if (p->var.generic) return set_error(FD_ERR_UNSUPPORTED, "the generic kernel has no variants");
    p->stores.clear();   // a stored forward's tables belong to the old variant
    int prefs[kMaxVariants];
    const int np = p->prob.dim == 2 ? variants_2d(p->shape_eff, p->st.M, prefs, kMaxVariants)
                                    : variants_3d(p->shape_eff, p->st.M, prefs, kMaxVariants);
    if (std::find(prefs, prefs + np, variant) == prefs + np)
        return set_error(FD_ERR_UNSUPPORTED, "variant %d is not built for this stencil", variant);
    if (p->prob.dim == 2 && z_chunk) return set_error(FD_ERR_ARG, "2D plans have no z-chunk");
    TuneChoice c{variant, z_chunk};
    if (p->prob.dim == 3 && z_chunk == 0) {
        Variant v;
        int st = select_variant_3d(p->shape_eff, p->st.M, p->st.N, p->pad[2], p->pad[1], p->pad[0], &v, variant);
        if (st) return set_error(st, "variant %d is not available", variant);
        apply_variant(p, v);
        return ensure_tuned(p);     // cost-model z-chunk
    }
    return apply_choice(p, c);
}

extern "C" int fd_plan_get_info(const fd_plan *p, fd_plan_info *info)
{
    clear_error();
    if (!p || !info) return set_error(FD_ERR_ARG, "NULL argument");
    for (int i = 0; i < 3; ++i) info->padded[i] = p->pad[i];
    info->pitch = p->pitch;
    info->n_orbits = (int)p->keys.size();
    info->kernel = (p->prob.dim * 100 + p->var.shape * 10) + (p->var.generic ? 1 : 0);
    info->courant_max = p->cmax;
    info->tile[0] = p->var.tx;
    info->tile[1] = p->var.tz;
    info->tile[2] = p->zchunk;
    info->effective_shape = p->shape_eff;
    return FD_OK;
}

extern "C" int fd_forward_workspace_size(const fd_plan *p, int nsrc, int nrec, size_t *bytes)
{
    clear_error();
    if (!p || !bytes || nsrc < 0 || nrec < 0) return set_error(FD_ERR_ARG, "bad argument");
    *bytes = make_layout(p, nsrc, nrec, false, 1).total;
    return FD_OK;
}

extern "C" int fd_gradient_workspace_size(const fd_plan *p, int nsrc, int nrec, int k, size_t *bytes)
{
    clear_error();
    if (!p || !bytes || nsrc < 0 || nrec < 0 || k < 1) return set_error(FD_ERR_ARG, "bad argument");
    *bytes = make_layout(p, nsrc, nrec, true, std::min(k, std::max(p->prob.nt, 1))).total;
    return FD_OK;
}

namespace {

int upload_tables(fd_plan *p, const Layout &L, char *ws, const Tables &T, cudaStream_t s)
{
    FDW_CK(cudaMemcpyAsync(ws + L.tab, T.blob.data(), T.blob.size(), cudaMemcpyHostToDevice, s));
    return FD_OK;
}

int upload_maps(fd_plan *p, const Layout &L, char *ws, int nbuf, cudaStream_t s)
{
    std::vector<CUtensorMap> maps(2 * nbuf + 1);
    for (int i = 0; i < nbuf; ++i)
        for (int t = 0; t < 2; ++t) {
            int r = encode_field_map(p, &maps[2 * i + t], reinterpret_cast<const float *>(ws + L.buf[i]),
                                     t == 1 && p->prob.dim == 3);
            if (r) return set_error(FD_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", r);
        }
    int r = encode_field_map(p, &maps[2 * nbuf], reinterpret_cast<const float *>(ws + L.kappa),
                             p->prob.dim == 3);
    if (r) return set_error(FD_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", r);
    FDW_CK(cudaMemcpyAsync(ws + L.tmaps, maps.data(), maps.size() * sizeof(CUtensorMap),
                           cudaMemcpyHostToDevice, s));
    return FD_OK;
}

// Instantiated time-loop graphs (single-shot and batched runs), keyed by
// workspace address, plan ids (never reused, unlike addresses), data
// pointers, sizes and kernel variant.  Every per-call state lives in the
// workspace and is re-initialised before a replay.  At most kGraphCache entries; evicting one synchronises
// the device first so that no launch of it is pending.
constexpr size_t kGraphCache = 8;
std::mutex g_graph_mu;
std::vector<std::pair<std::vector<uint64_t>, cudaGraphExec_t>> g_graphs;

cudaGraphExec_t graph_cache_find(const std::vector<uint64_t> &key)
{
    std::lock_guard<std::mutex> lock(g_graph_mu);
    for (auto &e : g_graphs)
        if (e.first == key) return e.second;
    return nullptr;
}

void graph_cache_put(const std::vector<uint64_t> &key, cudaGraphExec_t ge)
{
    std::lock_guard<std::mutex> lock(g_graph_mu);
    if (g_graphs.size() >= kGraphCache) {
        cudaDeviceSynchronize();
        cudaGraphExecDestroy(g_graphs.front().second);
        g_graphs.erase(g_graphs.begin());
    }
    g_graphs.emplace_back(key, ge);
}

// stride between consecutive z (rows in 2D, planes in 3D), in floats
int64_t zstride(const fd_plan *p) { return p->prob.dim == 3 ? p->plane : p->pitch; }

int prep_model(fd_plan *p, const Layout &L, char *ws, int kind, const float *model, cudaStream_t s)
{
    const fd_problem &pr = p->prob;
    const int64_t phys[3] = {pr.n[0], pr.n[1], pr.n[2]};
    const float vmax2 = (float)(pr.vmax * pr.vmax * (1.0 + 1e-6));
    FDW_CK(launch_prep_kappa(model, kind, reinterpret_cast<float *>(ws + L.kappa), pr.dim, phys,
                             pr.nb, p->pad, p->pitch, zstride(p), pr.dt / pr.h, vmax2,
                             reinterpret_cast<int *>(ws + L.status), s));
    return FD_OK;
}

}  // namespace

namespace {

// Copy a packed padded state [2][pad] into / out of two pitched buffers.
int state_in(fd_plan *p, const float *src, float *b0, float *b1, cudaStream_t s)
{
    const int64_t n = p->pad[0] * p->pad[1] * p->pad[2];
    FDW_CK(launch_copy_state(src, p->pad[2], p->pad[2] * p->pad[1], b0, p->pitch, zstride(p), p->pad, s));
    FDW_CK(launch_copy_state(src + n, p->pad[2], p->pad[2] * p->pad[1], b1, p->pitch, zstride(p), p->pad, s));
    return FD_OK;
}

int state_out(fd_plan *p, const float *b0, const float *b1, float *dst, cudaStream_t s)
{
    const int64_t n = p->pad[0] * p->pad[1] * p->pad[2];
    FDW_CK(launch_copy_state(b0, p->pitch, zstride(p), dst, p->pad[2], p->pad[2] * p->pad[1], p->pad, s));
    FDW_CK(launch_copy_state(b1, p->pitch, zstride(p), dst + n, p->pad[2], p->pad[2] * p->pad[1], p->pad, s));
    return FD_OK;
}

struct FwdBind {
    const PtEntry *inj, *smp;
    const int32_t *inj_ptr, *smp_ptr;
};

}  // namespace

namespace fdw {

int forward_impl(fd_plan *p, int model_kind, const float *model, int nsrc, const int64_t *src,
                 const float *wavelet, int nrec, const int64_t *rec, float *traces,
                 const float *state_in_d, float *state_out_d, void *ws, size_t ws_bytes,
                 void *stream, bool graphs)
{
    if (!p) return set_error(FD_ERR_ARG, "plan is NULL");
    const Layout L = make_layout(p, nsrc, nrec, false, 1);
    int st = check_common(p, model_kind, model, nsrc, src, wavelet, nrec, rec, ws, ws_bytes, L.total);
    if (st) return st;
    if (nrec > 0 && !traces) return set_error(FD_ERR_ARG, "traces is NULL");
    if ((st = ensure_tuned(p))) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *w = reinterpret_cast<char *>(ws);
    Tables T;
    if ((st = make_tables(p, nsrc, src, nrec, rec, false, T))) return st;
    if ((st = upload_tables(p, L, w, T, s))) return st;
    if ((st = upload_maps(p, L, w, 2, s))) return st;
    FDW_CK(cudaMemsetAsync(w + L.status, 0, kAlign, s));
    float *A = reinterpret_cast<float *>(w + L.buf[0]);
    float *B = reinterpret_cast<float *>(w + L.buf[1]);
    const size_t fb = (size_t)p->field * sizeof(float);
    FDW_CK(cudaMemsetAsync(A, 0, fb, s));
    FDW_CK(cudaMemsetAsync(B, 0, fb, s));
    if ((st = prep_model(p, L, w, model_kind, model, s))) return st;
    if (state_in_d && (st = state_in(p, state_in_d, A, B, s))) return st;
    const CUtensorMap *maps = reinterpret_cast<const CUtensorMap *>(w + L.tmaps);
    StepParams sp;
    fill_params(p, sp);
    sp.kappa = reinterpret_cast<const float *>(w + L.kappa);
    sp.status = reinterpret_cast<int *>(w + L.status);
    if (nsrc > 0) {
        sp.inj_ptr = reinterpret_cast<const int32_t *>(w + L.tab + T.inj_ptr);
        sp.inj = reinterpret_cast<const PtEntry *>(w + L.tab + T.inj);
        sp.inj_series = wavelet;
        sp.inj_ncol = nsrc;
    }
    if (nrec > 0) {
        sp.smp_ptr = reinterpret_cast<const int32_t *>(w + L.tab + T.smp_ptr);
        sp.smp = reinterpret_cast<const PtEntry *>(w + L.tab + T.smp);
        sp.smp_out = traces;
        sp.smp_ncol = nrec;
    }
    // Time loop: one cooperative persistent launch when asked for (small 2D
    // grids, FDWAVE_PERSISTENT=1), else one launch per step, captured once
    // into a CUDA graph per (workspace, plan, pointers, variant) and replayed
    // (FDWAVE_GRAPHS=0: plain launches).
    int pgrid = 0;
    {
        const char *e = getenv("FDWAVE_PERSISTENT");
        if (e && e[0] == '1' && p->prob.dim == 2 && p->prob.nt >= 16 && !p->var.generic)
            pgrid = persist2d_grid(p->var, p->ntiles);
    }
    auto step_loop = [&](cudaStream_t ls) -> cudaError_t {
        for (int n = 0; n < p->prob.nt; ++n) {
            const int cur = n & 1;
            bind_maps(sp, maps, 2, cur, cur ^ 1);
            sp.u_cur = cur ? B : A;
            sp.u_prev = cur ? A : B;
            sp.step = n;
            sp.check = check_step(n, p->prob.nt);
            cudaError_t e = launch(p, kModeForward, sp, ls);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    const bool hooked = debug_hook(p, sp);
    const char *ge_env = getenv("FDWAVE_GRAPHS");
    const bool use_graph = graphs && pgrid == 0 && p->prob.nt >= 16 && !(ge_env && ge_env[0] == '0') && !hooked;
    if (pgrid > 0) {
        PersistParams pp;
        std::memset(&pp, 0, sizeof pp);
        pp.base = sp;
        pp.maps = maps;
        pp.buf[0] = A;
        pp.buf[1] = B;
        pp.nt = p->prob.nt;
        int *stw = reinterpret_cast<int *>(w + L.status);
        pp.abort_flag = stw + 1;
        pp.bar_count = reinterpret_cast<unsigned int *>(stw + 2);
        pp.bar_gen = reinterpret_cast<unsigned int *>(stw + 3);
        FDW_CK(launch_persist2d(p->var, pp, pgrid, s));
    } else if (use_graph) {
        const std::vector<uint64_t> key = {
            1ull, reinterpret_cast<uint64_t>(ws), p->id,
            reinterpret_cast<uint64_t>(wavelet), reinterpret_cast<uint64_t>(traces),
            ((uint64_t)(uint32_t)nsrc << 32) | (uint32_t)nrec, (uint64_t)p->prob.nt,
            ((uint64_t)p->var.tz << 32) | (uint32_t)p->zchunk,
            ((uint64_t)p->var.threads << 32) | (uint32_t)p->var.generic};
        cudaGraphExec_t ge = nullptr;
        if (t_tune_graphs) {
            auto it = t_tune_graphs->find(key);
            if (it != t_tune_graphs->end()) ge = it->second;
        } else {
            ge = graph_cache_find(key);
        }
        if (!ge) {
            cudaStream_t cs;
            FDW_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            FDW_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            const cudaError_t ce = step_loop(cs);
            const cudaError_t ee = cudaStreamEndCapture(cs, &g);
            cudaStreamDestroy(cs);
            if (ce != cudaSuccess || ee != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return set_error(FD_ERR_CUDA, "graph capture failed: %s",
                                 cudaGetErrorString(ce != cudaSuccess ? ce : ee));
            }
            const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) return set_error(FD_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ie));
            if (t_tune_graphs) (*t_tune_graphs)[key] = ge;
            else graph_cache_put(key, ge);
        }
        FDW_CK(cudaGraphLaunch(ge, s));
    } else {
        FDW_CK(step_loop(s));
    }
    if (state_out_d) {
        const bool even = (p->prob.nt % 2) == 0;
        if ((st = state_out(p, even ? A : B, even ? B : A, state_out_d, s))) return st;
    }
    p->last_ws = ws;
    return FD_OK;
}

}  // namespace fdw

extern "C" int fd_forward(fd_plan *p, int model_kind, const float *model, int nsrc,
                          const int64_t *src, const float *wavelet, int nrec, const int64_t *rec,
                          float *traces, const float *state_in_d, float *state_out_d, void *ws,
                          size_t ws_bytes, void *stream)
{
    clear_error();
    if (p) forget_store(p, ws);
    return forward_impl(p, model_kind, model, nsrc, src, wavelet, nrec, rec, traces, state_in_d,
                        state_out_d, ws, ws_bytes, stream, true);
}

extern "C" int fd_status_read(const fd_plan *p, void *ws, void *stream)
{
    clear_error();
    if (!p || !ws) return set_error(FD_ERR_ARG, "NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int word = 0;
    FDW_CK(cudaMemcpyAsync(&word, ws, sizeof word, cudaMemcpyDeviceToHost, s));
    FDW_CK(cudaStreamSynchronize(s));
    FDW_CK(cudaMemsetAsync(ws, 0, sizeof word, s));
    if (word & kStatusTimeout) return set_error(FD_ERR_TIMEOUT, "a bounded device wait timed out");
    if (word & kStatusVmax)
        return set_error(FD_ERR_UNSTABLE, "model velocity exceeds the plan's vmax%s",
                         (word & kStatusBlowup) ? ", and the wavefield grew without bound" : "");
    if (word & kStatusBlowup)
        return set_error(FD_ERR_UNSTABLE, "the wavefield became non-finite or exceeded %g in "
                         "magnitude (checked every %d steps and at the last step)",
                         (double)kBlowupAmp, kCheckEvery);
    return FD_OK;
}

namespace {

// The checkpointed gradient in two phases: kGradForward sets the workspace up
// (tables, maps, kappa, cleared buffers) and runs the forward sweep; kGradAdjoint
// runs the backward sweep (restore and recompute per segment, unless one
// segment holds every D) and the fold.  fd_adjoint_gradient runs both;
// fd_gradient_forward and fd_gradient_adjoint run one each with k = nt.
constexpr int kGradForward = 1, kGradAdjoint = 2;

int gradient_run(fd_plan *p, int model_kind, const float *model, int nsrc, const int64_t *src,
                 const float *wavelet, int nrec, const int64_t *rec, const float *resid, int k,
                 float *grad, float *traces, float *wavelet_grad, void *ws, void *stream,
                 int phases)
{
    const int nt = p->prob.nt;
    const Layout L = make_layout(p, nsrc, nrec, true, k);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *w = reinterpret_cast<char *>(ws);
    int st = 0;
    Tables T;
    if ((st = make_tables(p, nsrc, src, nrec, rec, true, T))) return st;
    const size_t fb = up((size_t)p->field * sizeof(float));
    float *buf[4];
    for (int i = 0; i < 4; ++i) buf[i] = reinterpret_cast<float *>(w + L.buf[i]);
    float *gacc = reinterpret_cast<float *>(w + L.gacc);
    if (phases & kGradForward) {
        if ((st = upload_tables(p, L, w, T, s))) return st;
        if ((st = upload_maps(p, L, w, 4, s))) return st;
        FDW_CK(cudaMemsetAsync(w + L.status, 0, kAlign, s));
        for (int i = 0; i < 2; ++i) FDW_CK(cudaMemsetAsync(buf[i], 0, fb, s));
        if ((st = prep_model(p, L, w, model_kind, model, s))) return st;
    }
    if (phases & kGradAdjoint) {   // cleared here, so one stored forward serves several adjoints
        for (int i = 2; i < 4; ++i) FDW_CK(cudaMemsetAsync(buf[i], 0, fb, s));
        FDW_CK(cudaMemsetAsync(gacc, 0, fb, s));
    }
    const CUtensorMap *maps = reinterpret_cast<const CUtensorMap *>(w + L.tmaps);
    char *ck = w + L.ckpt;
    char *dseg = w + L.dseg;

    StepParams sp;
    fill_params(p, sp);
    debug_hook(p, sp);
    sp.kappa = reinterpret_cast<const float *>(w + L.kappa);
    sp.status = reinterpret_cast<int *>(w + L.status);
    auto bind_fwd = [&](bool sample) {
        sp.inj_ptr = nsrc ? reinterpret_cast<const int32_t *>(w + L.tab + T.inj_ptr) : nullptr;
        sp.inj = reinterpret_cast<const PtEntry *>(w + L.tab + T.inj);
        sp.inj_series = wavelet;
        sp.inj_ncol = nsrc;
        sp.smp_ptr = (sample && nrec && traces) ? reinterpret_cast<const int32_t *>(w + L.tab + T.smp_ptr) : nullptr;
        sp.smp = reinterpret_cast<const PtEntry *>(w + L.tab + T.smp);
        sp.smp_out = traces;
        sp.smp_ncol = nrec;
    };
    // One segment (k >= nt: D of every step fits the workspace, e.g. 124 GB for
    // 296^3 x 1200 steps): the forward sweep itself stores D, and there is no
    // checkpoint and no recompute (48 instead of 64 + 32/k bytes per point and
    // step).  The store-D mode rounds exactly like the forward mode, so the
    // result is bitwise that of any checkpoint interval.
    const bool store_all = L.nck == 1;
    // forward sweep with checkpoints (u^n, u^{n-1}) at n = s k
    bind_fwd(true);
    for (int n = 0; n < ((phases & kGradForward) ? nt : 0); ++n) {
        const int cur = n & 1;
        if (n % k == 0 && !store_all) {
            const int c = n / k;
            FDW_CK(cudaMemcpyAsync(ck + (size_t)(2 * c) * fb, buf[cur], fb, cudaMemcpyDeviceToDevice, s));
            FDW_CK(cudaMemcpyAsync(ck + (size_t)(2 * c + 1) * fb, buf[cur ^ 1], fb, cudaMemcpyDeviceToDevice, s));
        }
        bind_maps(sp, maps, 4, cur, cur ^ 1);
        sp.u_cur = buf[cur];
        sp.u_prev = buf[cur ^ 1];
        sp.step = n;
        sp.check = check_step(n, nt);
        sp.dseg_out = store_all ? reinterpret_cast<float *>(dseg + (size_t)n * fb) : nullptr;
        FDW_CK(launch(p, store_all ? kModeStoreD : kModeForward, sp, s));
    }
    sp.dseg_out = nullptr;
    if (!(phases & kGradAdjoint)) return FD_OK;
    // backward sweep over segments
    int t = 0;   // adjoint steps done: q^{j+1} lives in buf[2 + (t & 1)]
    for (int c = L.nck - 1; c >= 0; --c) {
        const int k0 = c * k, k1 = std::min(k0 + k, nt);
        bind_fwd(false);
        if (!store_all) {
            FDW_CK(cudaMemcpyAsync(buf[0], ck + (size_t)(2 * c) * fb, fb, cudaMemcpyDeviceToDevice, s));
            FDW_CK(cudaMemcpyAsync(buf[1], ck + (size_t)(2 * c + 1) * fb, fb, cudaMemcpyDeviceToDevice, s));
            for (int n = k0; n < k1; ++n) {
                const int cur = (n - k0) & 1;
                bind_maps(sp, maps, 4, cur, cur ^ 1);
                sp.u_cur = buf[cur];
                sp.u_prev = buf[cur ^ 1];
                sp.step = n;
                sp.check = 0;   // the recompute repeats the checked forward sweep bit for bit
                sp.dseg_out = reinterpret_cast<float *>(dseg + (size_t)(n - k0) * fb);
                FDW_CK(launch(p, kModeStoreD, sp, s));
            }
        }
        sp.dseg_out = nullptr;
        sp.inj_ptr = nrec ? reinterpret_cast<const int32_t *>(w + L.tab + T.ainj_ptr) : nullptr;
        sp.inj = reinterpret_cast<const PtEntry *>(w + L.tab + T.ainj);
        sp.inj_series = resid;
        sp.inj_ncol = nrec;
        sp.smp_ptr = (nsrc && wavelet_grad) ? reinterpret_cast<const int32_t *>(w + L.tab + T.asmp_ptr) : nullptr;
        sp.smp = reinterpret_cast<const PtEntry *>(w + L.tab + T.asmp);
        sp.smp_out = wavelet_grad;
        sp.smp_ncol = nsrc;
        sp.gacc = gacc;
        for (int j = k1; j > k0; --j, ++t) {
            const int cur = 2 + (t & 1);
            bind_maps(sp, maps, 4, cur, cur ^ 1);
            sp.u_cur = buf[cur];
            sp.u_prev = buf[cur ^ 1];
            sp.step = j - 1;
            sp.check = check_step(t, nt);
            sp.dseg_in = reinterpret_cast<const float *>(dseg + (size_t)(j - 1 - k0) * fb);
            FDW_CK(launch(p, kModeAdjoint, sp, s));
        }
        sp.gacc = nullptr;
        sp.dseg_in = nullptr;
    }
    const fd_problem &pr = p->prob;
    const int64_t phys[3] = {pr.n[0], pr.n[1], pr.n[2]};
    FDW_CK(launch_fold_grad(gacc, p->pitch, zstride(p), phys, pr.nb, (float)(-1.0 / (pr.dt * pr.dt)),
                            grad, s));
    return FD_OK;
}

}  // namespace

extern "C" int fd_adjoint_gradient(fd_plan *p, int model_kind, const float *model, int nsrc,
                                   const int64_t *src, const float *wavelet, int nrec,
                                   const int64_t *rec, const float *resid, int k, float *grad,
                                   float *traces, float *wavelet_grad, void *ws, size_t ws_bytes,
                                   void *stream)
{
    clear_error();
    if (!p) return set_error(FD_ERR_ARG, "plan is NULL");
    if (k < 1) return set_error(FD_ERR_ARG, "ckpt_every must be >= 1");
    k = std::min(k, std::max(p->prob.nt, 1));
    const Layout L = make_layout(p, nsrc, nrec, true, k);
    int st = check_common(p, model_kind, model, nsrc, src, wavelet, nrec, rec, ws, ws_bytes, L.total);
    if (st) return st;
    if (!grad) return set_error(FD_ERR_ARG, "grad is NULL");
    if (nrec > 0 && !resid) return set_error(FD_ERR_ARG, "resid is NULL");
    if ((st = ensure_tuned(p))) return st;
    forget_store(p, ws);
    st = gradient_run(p, model_kind, model, nsrc, src, wavelet, nrec, rec, resid, k, grad, traces,
                      wavelet_grad, ws, stream, kGradForward | kGradAdjoint);
    if (st) return st;
    p->last_ws = ws;
    return FD_OK;
}

extern "C" int fd_gradient_forward(fd_plan *p, int model_kind, const float *model, int nsrc,
                                   const int64_t *src, const float *wavelet, int nrec,
                                   const int64_t *rec, float *traces, void *ws, size_t ws_bytes,
                                   void *stream)
{
    clear_error();
    if (!p) return set_error(FD_ERR_ARG, "plan is NULL");
    const int k = std::max(p->prob.nt, 1);
    const Layout L = make_layout(p, nsrc, nrec, true, k);
    int st = check_common(p, model_kind, model, nsrc, src, wavelet, nrec, rec, ws, ws_bytes, L.total);
    if (st) return st;
    if ((st = ensure_tuned(p))) return st;
    forget_store(p, ws);
    st = gradient_run(p, model_kind, model, nsrc, src, wavelet, nrec, rec, nullptr, k, nullptr, traces,
                      nullptr, ws, stream, kGradForward);
    if (st) return st;
    p->stores.push_back({ws, points_hash(nsrc, src, nrec, rec)});
    if (p->stores.size() > 64) p->stores.erase(p->stores.begin());
    p->last_ws = ws;
    return FD_OK;
}

extern "C" int fd_gradient_adjoint(fd_plan *p, int nsrc, const int64_t *src, int nrec,
                                   const int64_t *rec, const float *resid, float *grad,
                                   float *wavelet_grad, void *ws, size_t ws_bytes, void *stream)
{
    clear_error();
    if (!p) return set_error(FD_ERR_ARG, "plan is NULL");
    if (nsrc < 0 || nrec < 0 || (nsrc > 0 && !src) || (nrec > 0 && !rec))
        return set_error(FD_ERR_ARG, "bad source or receiver arguments");
    const uint64_t h = points_hash(nsrc, src, nrec, rec);
    bool known = false;
    for (const auto &e : p->stores) known = known || (e.first == ws && e.second == h);
    if (!ws || !known)
        return set_error(FD_ERR_ARG, "no fd_gradient_forward of this plan with this workspace and "
                         "these sources and receivers precedes the call");
    const int k = std::max(p->prob.nt, 1);
    const Layout L = make_layout(p, nsrc, nrec, true, k);
    if (ws_bytes < L.total) return set_error(FD_ERR_NOMEM, "workspace has %zu bytes, needs %zu", ws_bytes, L.total);
    if (!grad) return set_error(FD_ERR_ARG, "grad is NULL");
    if (nrec > 0 && !resid) return set_error(FD_ERR_ARG, "resid is NULL");
    int st = gradient_run(p, FD_MODEL_VELOCITY, nullptr, nsrc, src, nullptr, nrec, rec, resid, k, grad,
                          nullptr, wavelet_grad, ws, stream, kGradAdjoint);
    if (st) return st;
    p->last_ws = ws;
    return FD_OK;
}

// ------------------------------ batched shots ------------------------------
// 2D shots sharing a specialised stencil run as one launch per time step over
// a tile table spanning every shot (step2d_batched); other batches launch the
// step kernel of each shot in turn.  Either way the whole time loop is
// captured once into a CUDA graph and replayed.

namespace {

// Common batch variant for 2D shots (nullptr if the batch needs per-shot launches).
// Tile rows per thread chosen for a batch by fd_forward_batched_autotune,
// keyed by device, stencil, shot count and total padded points.
std::mutex g_batch_mu;
std::map<std::string, int> g_batch_tune;

std::string batch_key(int nshots, const fd_shot *shots)
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, dev);
    int64_t pts = 0;
    for (int i = 0; i < nshots; ++i) pts += shots[i].plan->pad[0] * shots[i].plan->pad[2];
    const fd_plan *p0 = shots[0].plan;
    char buf[256];
    snprintf(buf, sizeof buf, "%s|batch|%d|%d|%d|%lld", prop.name, p0->shape_eff, p0->st.M, nshots,
             (long long)pts);
    return buf;
}

int batch_choice(int nshots, const fd_shot *shots)
{
    std::lock_guard<std::mutex> lock(g_batch_mu);
    auto it = g_batch_tune.find(batch_key(nshots, shots));
    return it == g_batch_tune.end() ? 0 : it->second;
}

// Common single-launch variant of a 2D batch with R rows per thread (0: the
// tuned or default choice); false if the batch needs per-shot launches.
bool batch_geometry(int nshots, const fd_shot *shots, Variant &bv, std::vector<TileGeo> &geo,
                    int R = 0)
{
    const fd_plan *p0 = shots[0].plan;
    if (p0->prob.dim != 2 || p0->var.generic) return false;
    int64_t tiles4 = 0;
    for (int i = 0; i < nshots; ++i) {
        const fd_plan *q = shots[i].plan;
        if (q->shape_eff != p0->shape_eff || q->st.M != p0->st.M || q->var.generic) return false;
        tiles4 += ((q->pad[2] + 63) / 64) * ((q->pad[0] + 63) / 64);
    }
    if (R == 0) R = batch_choice(nshots, shots);
    if (batch2d_variant(p0->shape_eff, p0->st.M, tiles4, &bv, R)) return false;
    geo.resize(nshots);
    for (int i = 0; i < nshots; ++i) {
        const fd_plan *q = shots[i].plan;
        const int tx = (int)((q->pad[2] + bv.tx - 1) / bv.tx), tz = (int)((q->pad[0] + bv.tz - 1) / bv.tz);
        geo[i] = {bv.tx, bv.tz, tx, tx * tz};
    }
    return true;
}

// Extra workspace of a single-launch batch: descriptors, tile records and,
// when the two-step kernel supports the stencil, two more field buffers per
// shot and the extended-region source table (a source lies in at most four
// tiles' extended regions).
size_t batch_extra_bytes(int nshots, const fd_shot *shots, int64_t ntiles, bool two)
{
    size_t b = up(nshots * sizeof(ShotDesc)) + up(ntiles * sizeof(TileRec));
    if (two) {
        int64_t nsrc = 0;
        for (int i = 0; i < nshots; ++i) {
            b += 2 * up(shots[i].plan->field * sizeof(float));
            nsrc += shots[i].nsrc;
        }
        b += up(std::max<int64_t>(4 * nsrc, 1) * sizeof(PtEntry));
    }
    return b;
}

// The two-step kernel applies to single-launch batches of its stencils with at
// least two steps, when FDWAVE_BATCH_2STEP=1 (opt-in: on the 48-shot Cross(4)
// workload it measured 187 Gpts/s against 250 for the one-step kernel, whose
// pass is not bound by HBM alone).
bool batch_two_step(const fd_plan *p0, bool one, Batch2Geo *g)
{
    if (!one || p0->prob.nt < 2 || batch2d2_geometry(p0->shape_eff, p0->st.M, g) != FD_OK)
        return false;
    const char *e = std::getenv("FDWAVE_BATCH_2STEP");
    return e && std::strcmp(e, "1") == 0;
}

}  // namespace

namespace {

// Workspace of a batch laid out for tile rows R (0: the tuned or default R).
size_t batch_bytes(int nshots, const fd_shot *shots, int R)
{
    size_t tot = 0;
    Variant bv;
    std::vector<TileGeo> geo;
    const bool one = nshots > 0 && batch_geometry(nshots, shots, bv, geo, R);
    int64_t ntiles = 0;
    for (int i = 0; i < nshots; ++i) {
        const int nt_tab = one ? geo[i].ntiles : -1;
        tot += make_layout(shots[i].plan, shots[i].nsrc, shots[i].nrec, false, 1, nt_tab).total;
        if (one) ntiles += geo[i].ntiles;
    }
    Batch2Geo g2;
    const bool two = nshots > 0 && batch_two_step(shots[0].plan, one, &g2);
    if (one) tot += batch_extra_bytes(nshots, shots, ntiles, two);
    return tot;
}

}  // namespace

extern "C" int fd_forward_batched_workspace_size(int nshots, const fd_shot *shots, size_t *bytes)
{
    clear_error();
    if (nshots < 0 || (nshots > 0 && !shots) || !bytes) return set_error(FD_ERR_ARG, "bad argument");
    for (int i = 0; i < nshots; ++i)
        if (!shots[i].plan) return set_error(FD_ERR_ARG, "shot %d has no plan", i);
    // enough for every tile shape the batch can take (the tuned one included)
    size_t tot = batch_bytes(nshots, shots, 2);
    if (nshots > 0) {
        int rs[4];
        const int nr = batch2d_variants(shots[0].plan->shape_eff, shots[0].plan->st.M, rs, 4);
        for (int i = 0; i < nr; ++i) tot = std::max(tot, batch_bytes(nshots, shots, rs[i]));
    }
    *bytes = tot;
    return FD_OK;
}

namespace {

int forward_batched_impl(int nshots, const fd_shot *shots, void *ws, size_t ws_bytes, void *stream,
                         int R, bool graphs)
{
    size_t need = 0;
    int st = fd_forward_batched_workspace_size(nshots, shots, &need);
    if (st) return st;
    if (!ws || ws_bytes < need) return set_error(FD_ERR_NOMEM, "workspace too small (%zu < %zu)", ws_bytes, need);
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return set_error(FD_ERR_ARG, "workspace must be 256-byte aligned");
    if (nshots == 0) return FD_OK;
    const fd_plan *p0 = shots[0].plan;
    for (int i = 1; i < nshots; ++i) {
        const fd_plan *q = shots[i].plan;
        if (q->prob.dim != p0->prob.dim || q->prob.nt != p0->prob.nt || q->prob.dt != p0->prob.dt ||
            q->st.M != p0->st.M || q->st.shape != p0->st.shape || q->st.scheme != p0->st.scheme ||
            std::memcmp(q->W, p0->W, sizeof q->W) != 0)
            return set_error(FD_ERR_ARG, "shot %d: batched shots must share dim, stencil, dt and nt", i);
    }
    Variant bv;
    std::vector<TileGeo> geo;
    bool one = batch_geometry(nshots, shots, bv, geo, R);
    Batch2Geo g2;
    const bool two = batch_two_step(p0, one, &g2);
    if (two && bv.tz != g2.tz) one = batch_geometry(nshots, shots, bv, geo, g2.tz / 16);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *base = reinterpret_cast<char *>(ws);
    // extra region (after every shot's slice): descriptors | tile records |
    // two-step buffers of each shot | extended-region source table
    int64_t ntiles_all = 0;
    size_t shots_bytes = 0;
    for (int i = 0; i < nshots; ++i) {
        shots_bytes += make_layout(shots[i].plan, shots[i].nsrc, shots[i].nrec, false, 1,
                                   one ? geo[i].ntiles : -1).total;
        if (one) ntiles_all += geo[i].ntiles;
    }
    char *extra = base + shots_bytes;
    char *xbufs = extra + up(nshots * sizeof(ShotDesc)) + up(ntiles_all * sizeof(TileRec));
    char *xtab = xbufs;
    if (two)
        for (int i = 0; i < nshots; ++i) xtab += 2 * up(shots[i].plan->field * sizeof(float));
    std::vector<PtEntry> ext;
    std::vector<StepParams> sps(one ? 0 : nshots);
    std::vector<ShotDesc> descs(one ? nshots : 0);
    std::vector<TileRec> recs;
    std::vector<float *> As(nshots), Bs(nshots);
    std::vector<const CUtensorMap *> mp(nshots);
    for (int i = 0; i < nshots; ++i) {
        fd_plan *p = const_cast<fd_plan *>(shots[i].plan);
        const fd_shot &sh = shots[i];
        const Layout L = make_layout(p, sh.nsrc, sh.nrec, false, 1, one ? geo[i].ntiles : -1);
        st = check_common(p, sh.model_kind, sh.model_d, sh.nsrc, sh.src_idx, sh.wavelet_d, sh.nrec,
                          sh.rec_idx, base, L.total, L.total);
        if (st) return set_error(st, "shot %d: %s", i, fd_last_error());
        if (sh.nrec > 0 && !sh.traces_d) return set_error(FD_ERR_ARG, "shot %d: traces is NULL", i);
        if ((st = ensure_tuned(p))) return st;
        Tables T;
        if ((st = make_tables(p, sh.nsrc, sh.src_idx, sh.nrec, sh.rec_idx, false, T,
                              one ? &geo[i] : nullptr)))
            return st;
        if ((st = upload_tables(p, L, base, T, s))) return st;
        FDW_CK(cudaMemsetAsync(base + L.status, 0, kAlign, s));
        As[i] = reinterpret_cast<float *>(base + L.buf[0]);
        Bs[i] = reinterpret_cast<float *>(base + L.buf[1]);
        FDW_CK(cudaMemsetAsync(As[i], 0, (size_t)p->field * 4, s));
        FDW_CK(cudaMemsetAsync(Bs[i], 0, (size_t)p->field * 4, s));
        if ((st = prep_model(p, L, base, sh.model_kind, sh.model_d, s))) return st;
        const int32_t *ip = reinterpret_cast<const int32_t *>(base + L.tab + T.inj_ptr);
        const PtEntry *ie = reinterpret_cast<const PtEntry *>(base + L.tab + T.inj);
        const int32_t *sp_ = reinterpret_cast<const int32_t *>(base + L.tab + T.smp_ptr);
        const PtEntry *se = reinterpret_cast<const PtEntry *>(base + L.tab + T.smp);
        if (one) {
            ShotDesc &d = descs[i];
            std::memset(&d, 0, sizeof d);
            Variant keep = p->var;
            p->var = bv;     // maps with the batch's box
            const float *kap = reinterpret_cast<const float *>(base + L.kappa);
            int r = encode_field_map(p, &d.tmap[0], As[i], false);
            r = r ? r : encode_field_map(p, &d.tmap[1], Bs[i], false);
            r = r ? r : encode_field_map(p, &d.tile[0], As[i], true);
            r = r ? r : encode_field_map(p, &d.tile[1], Bs[i], true);
            r = r ? r : encode_field_map(p, &d.ktile, kap, true);
            p->var = keep;
            if (r) return set_error(FD_ERR_CUDA, "cuTensorMapEncodeTiled failed");
            if (two) {
                float *f2 = reinterpret_cast<float *>(xbufs);
                float *f3 = reinterpret_cast<float *>(xbufs + up(p->field * sizeof(float)));
                xbufs += 2 * up(p->field * sizeof(float));
                FDW_CK(cudaMemsetAsync(f2, 0, (size_t)p->field * 4, s));
                FDW_CK(cudaMemsetAsync(f3, 0, (size_t)p->field * 4, s));
                d.info.buf[2] = f2;
                d.info.buf[3] = f3;
                const float *bufs[4] = {As[i], Bs[i], f2, f3};
                const int64_t dims[2] = {p->pad[2], p->pad[0]};
                const int64_t str[1] = {p->pitch * 4};
                for (int b = 0; b < 4 && !r; ++b) {
                    r = encode_tmap(&d.c2[b], bufs[b], 2, dims, str, g2.cbox);
                    r = r ? r : encode_tmap(&d.p2[b], bufs[b], 2, dims, str, g2.pbox);
                }
                r = r ? r : encode_tmap(&d.k2, kap, 2, dims, str, g2.pbox);
                if (r) return set_error(FD_ERR_CUDA, "cuTensorMapEncodeTiled failed");
            }
            d.info.buf[0] = As[i];
            d.info.buf[1] = Bs[i];
            d.info.kappa = reinterpret_cast<const float *>(base + L.kappa);
            d.info.inj_ptr = sh.nsrc ? ip : nullptr;
            d.info.inj = ie;
            d.info.inj_series = sh.wavelet_d;
            d.info.inj_ncol = sh.nsrc;
            d.info.smp_ptr = sh.nrec ? sp_ : nullptr;
            d.info.smp = se;
            d.info.smp_out = sh.traces_d;
            d.info.smp_ncol = sh.nrec;
            d.info.nx = p->pad[2];
            d.info.nz = p->pad[0];
            d.info.pitch = p->pitch;
            d.info.phys_lo[0] = p->prob.nb; d.info.phys_hi[0] = p->prob.nb + p->prob.n[2] - 1;
            d.info.phys_lo[2] = p->prob.nb; d.info.phys_hi[2] = p->prob.nb + p->prob.n[0] - 1;
            d.info.gcoef = p->gcoef;
            d.info.tiles_x = geo[i].tiles_x;
            d.info.field = p->field;
            const int32_t *hip = reinterpret_cast<const int32_t *>(T.blob.data() + T.inj_ptr);
            const int32_t *hsp = reinterpret_cast<const int32_t *>(T.blob.data() + T.smp_ptr);
            // sources of each tile's extended region (tile plus the halo whose
            // u^{n+1} the two-step kernel computes), x relative to its origin
            std::vector<std::vector<PtEntry>> xt(two ? geo[i].ntiles : 0);
            if (two) {
                const fd_problem &pr = p->prob;
                const float sc = (float)(pr.dt * pr.dt / std::pow(pr.h, pr.dim));
                const int ntx = geo[i].tiles_x, ntz = geo[i].ntiles / ntx;
                for (int k = 0; k < sh.nsrc; ++k) {
                    const int64_t z = sh.src_idx[k] / pr.n[2] + pr.nb, x = sh.src_idx[k] % pr.n[2] + pr.nb;
                    for (int tz = 0; tz < ntz; ++tz)
                        for (int tx = 0; tx < ntx; ++tx) {
                            const int64_t ex0 = (int64_t)tx * geo[i].tx - g2.hx, ez0 = (int64_t)tz * geo[i].tz - p->st.M;
                            if (x < ex0 || x >= ex0 + geo[i].tx + 2 * g2.hx || z < ez0 ||
                                z >= ez0 + geo[i].tz + 2 * p->st.M)
                                continue;
                            PtEntry e;
                            e.z = (int32_t)z;
                            e.yx = (int32_t)(x - ex0);
                            e.col = k;
                            e.scale = sc;
                            xt[tz * ntx + tx].push_back(e);
                        }
                }
                for (auto &v : xt)
                    std::stable_sort(v.begin(), v.end(), [](const PtEntry &a, const PtEntry &b) { return a.z < b.z; });
            }
            for (int t = 0; t < geo[i].ntiles; ++t) {
                TileRec r;
                std::memset(&r, 0, sizeof r);
                r.shot = i;
                r.tile = t;
                if (two) {
                    r.xb = (int)ext.size();
                    ext.insert(ext.end(), xt[t].begin(), xt[t].end());
                    r.xe = (int)ext.size();
                }
                r.x0 = (t % geo[i].tiles_x) * geo[i].tx;
                r.z0 = (t / geo[i].tiles_x) * geo[i].tz;
                r.ib = sh.nsrc ? hip[t] : 0;
                r.ie = sh.nsrc ? hip[t + 1] : 0;
                r.sb = sh.nrec ? hsp[t] : 0;
                r.se = sh.nrec ? hsp[t + 1] : 0;
                recs.push_back(r);
            }
        } else {
            if ((st = upload_maps(p, L, base, 2, s))) return st;
            StepParams &sp = sps[i];
            fill_params(p, sp);
            sp.kappa = reinterpret_cast<const float *>(base + L.kappa);
            sp.status = reinterpret_cast<int *>(base + L.status);
            if (sh.nsrc > 0) {
                sp.inj_ptr = ip; sp.inj = ie; sp.inj_series = sh.wavelet_d; sp.inj_ncol = sh.nsrc;
            }
            if (sh.nrec > 0) {
                sp.smp_ptr = sp_; sp.smp = se; sp.smp_out = sh.traces_d; sp.smp_ncol = sh.nrec;
            }
            mp[i] = reinterpret_cast<const CUtensorMap *>(base + L.tmaps);
        }
        base += L.total;
    }
    BatchParams bp;
    std::memset(&bp, 0, sizeof bp);
    const int ntiles = (int)recs.size();
    if (one) {
        char *d = base;
        FDW_CK(cudaMemcpyAsync(d, descs.data(), nshots * sizeof(ShotDesc), cudaMemcpyHostToDevice, s));
        char *t1 = d + up(nshots * sizeof(ShotDesc));
        FDW_CK(cudaMemcpyAsync(t1, recs.data(), ntiles * sizeof(TileRec), cudaMemcpyHostToDevice, s));
        bp.shots = reinterpret_cast<const ShotDesc *>(d);
        bp.tiles = reinterpret_cast<const TileRec *>(t1);
        if (two && !ext.empty())
            FDW_CK(cudaMemcpyAsync(xtab, ext.data(), ext.size() * sizeof(PtEntry), cudaMemcpyHostToDevice, s));
        bp.ext = reinterpret_cast<const PtEntry *>(xtab);
        bp.ntiles = ntiles;
        // shot 0's status word collects the device conditions of the batch
        bp.status = reinterpret_cast<int *>(ws);
        std::memcpy(bp.w, p0->W, sizeof bp.w);
    }
    // The time loop is captured once per (workspace, shots) configuration and
    // replayed on later calls; all per-call state (models, tables, fields) is
    // re-initialised above, outside the graph.
    std::vector<uint64_t> key;
    key.push_back(reinterpret_cast<uint64_t>(ws));
    key.push_back((uint64_t)nshots);
    for (int i = 0; i < nshots; ++i) {
        const fd_shot &sh = shots[i];
        key.push_back(sh.plan->id);
        key.push_back(reinterpret_cast<uint64_t>(sh.wavelet_d));
        key.push_back(reinterpret_cast<uint64_t>(sh.traces_d));
        key.push_back(((uint64_t)(uint32_t)sh.nsrc << 32) | (uint32_t)sh.nrec);
    }
    key.push_back(two ? 1ull : 0ull);
    key.push_back(((uint64_t)bv.tz << 32) | (uint32_t)p0->prob.nt);
    key.insert(key.begin(), 2ull);
    {   // every step in one persistent launch (opt-in: FDWAVE_BATCH_PERSISTENT=1)
        const char *e = std::getenv("FDWAVE_BATCH_PERSISTENT");
        if (e && e[0] == '1' && one && !two) {
            FDW_CK(launch_batched2d_persistent(bv, bp, ntiles, p0->prob.nt, s));
            return FD_OK;
        }
    }
    if (!graphs) {   // launches one by one (autotuning: candidates with other nt or tiles)
        cudaError_t ce = cudaSuccess;
        const int nt = p0->prob.nt;
        for (int n = 0; n < nt && ce == cudaSuccess; ++n) {
            if (one) {
                bp.step = n;
                bp.parity = n & 1;
                bp.check = check_step(n, nt);
                ce = launch_batched2d(bv, bp, ntiles, s);
                continue;
            }
            for (int i = 0; i < nshots && ce == cudaSuccess; ++i) {
                StepParams &sp = sps[i];
                const int cur = n & 1;
                bind_maps(sp, mp[i], 2, cur, cur ^ 1);
                sp.u_cur = cur ? Bs[i] : As[i];
                sp.u_prev = cur ? As[i] : Bs[i];
                sp.step = n;
                sp.check = check_step(n, nt);
                ce = launch(shots[i].plan, kModeForward, sp, s);
            }
        }
        if (ce != cudaSuccess) return set_error(FD_ERR_CUDA, "batched launch failed: %s", cudaGetErrorString(ce));
        return FD_OK;
    }
    cudaGraphExec_t ge = graph_cache_find(key);
    if (!ge) {
        cudaStream_t cs;
        FDW_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        FDW_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        cudaError_t ce = cudaSuccess;
        const int nt = p0->prob.nt;
        if (two) {
            // an odd first step runs alone; then pairs of steps, the outputs
            // going to the pair of buffers not being read
            int n = 0, cur = 0, prev = 1;
            if (nt & 1) {
                bp.step = 0;
                bp.parity = 0;
                bp.check = check_step(0, nt);
                ce = launch_batched2d(bv, bp, ntiles, cs);
                n = 1; cur = 1; prev = 0;
            }
            for (; n + 1 < nt && ce == cudaSuccess; n += 2) {
                const int o1 = cur < 2 ? 2 : 0, o2 = o1 + 1;
                bp.roles[0] = cur; bp.roles[1] = prev; bp.roles[2] = o1; bp.roles[3] = o2;
                bp.step = n;
                bp.check = check_step(n, nt) || check_step(n + 1, nt);
                ce = launch_batched2d2(bv, bp, ntiles, cs);
                cur = o2; prev = o1;
            }
        }
        for (int n = 0; n < nt && ce == cudaSuccess && !two; ++n) {
            if (one) {
                bp.step = n;
                bp.parity = n & 1;
                bp.check = check_step(n, nt);
                ce = launch_batched2d(bv, bp, ntiles, cs);
                continue;
            }
            for (int i = 0; i < nshots && ce == cudaSuccess; ++i) {
                StepParams &sp = sps[i];
                const int cur = n & 1;
                bind_maps(sp, mp[i], 2, cur, cur ^ 1);
                sp.u_cur = cur ? Bs[i] : As[i];
                sp.u_prev = cur ? As[i] : Bs[i];
                sp.step = n;
                sp.check = check_step(n, nt);
                ce = launch(shots[i].plan, kModeForward, sp, cs);
            }
        }
        cudaError_t ee = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        if (ce != cudaSuccess || ee != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return set_error(FD_ERR_CUDA, "graph capture failed: %s",
                             cudaGetErrorString(ce != cudaSuccess ? ce : ee));
        }
        cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) return set_error(FD_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ie));
        graph_cache_put(key, ge);
    }
    FDW_CK(cudaGraphLaunch(ge, s));
    return FD_OK;
}

}  // namespace

extern "C" int fd_forward_batched(int nshots, const fd_shot *shots, void *ws, size_t ws_bytes,
                                  void *stream)
{
    clear_error();
    return forward_batched_impl(nshots, shots, ws, ws_bytes, stream, 0, true);
}

extern "C" int fd_forward_batched_set_variant(int nshots, const fd_shot *shots, int rows)
{
    clear_error();
    if (nshots < 1 || !shots) return set_error(FD_ERR_ARG, "bad argument");
    for (int i = 0; i < nshots; ++i)
        if (!shots[i].plan) return set_error(FD_ERR_ARG, "shot %d has no plan", i);
    int rs[4];
    const int nr = batch2d_variants(shots[0].plan->shape_eff, shots[0].plan->st.M, rs, 4);
    if (std::find(rs, rs + nr, rows) == rs + nr)
        return set_error(FD_ERR_UNSUPPORTED, "no batched kernel with %d rows per thread for this stencil", rows);
    std::lock_guard<std::mutex> lock(g_batch_mu);
    g_batch_tune[batch_key(nshots, shots)] = rows;
    return FD_OK;
}

extern "C" int fd_forward_batched_autotune(int nshots, const fd_shot *shots, void *ws, size_t ws_bytes,
                                           void *stream)
{
    clear_error();
    size_t need = 0;
    int st = fd_forward_batched_workspace_size(nshots, shots, &need);
    if (st) return st;
    if (!ws || ws_bytes < need) return set_error(FD_ERR_NOMEM, "workspace too small (%zu < %zu)", ws_bytes, need);
    if (nshots == 0) return FD_OK;
    Variant bv;
    std::vector<TileGeo> geo;
    if (!batch_geometry(nshots, shots, bv, geo, 2)) return FD_OK;   // per-shot launches: nothing to choose
    int rs[4];
    const int nr = batch2d_variants(shots[0].plan->shape_eff, shots[0].plan->st.M, rs, 4);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // candidates run on copies of the plans with 16 and 64 steps, launched one
    // by one (no graph); time per step = (best of 3 at 64 - best of 3 at 16) / 48
    std::vector<fd_plan> copies(nshots);
    std::vector<fd_shot> cs(shots, shots + nshots);
    for (int i = 0; i < nshots; ++i) {
        copies[i] = *shots[i].plan;
        cs[i].plan = &copies[i];
    }
    cudaEvent_t e0, e1;
    FDW_CK(cudaEventCreate(&e0));
    FDW_CK(cudaEventCreate(&e1));
    auto timed = [&](int R, int nt, float &out) -> int {
        for (auto &c : copies) c.prob.nt = nt;
        out = 1e30f;
        for (int r = 0; r < 3; ++r) {
            FDW_CK(cudaEventRecord(e0, s));
            const int rc = forward_batched_impl(nshots, cs.data(), ws, ws_bytes, stream, R, false);
            if (rc) return rc;
            FDW_CK(cudaEventRecord(e1, s));
            FDW_CK(cudaEventSynchronize(e1));
            float t = 0.f;
            FDW_CK(cudaEventElapsedTime(&t, e0, e1));
            out = std::min(out, t);
        }
        return FD_OK;
    };
    float best = 1e30f;
    int bestR = rs[0];
    for (int i = 0; i < nr && !st; ++i) {
        float t64 = 0.f, t16 = 0.f;
        if ((st = timed(rs[i], 64, t64)) || (st = timed(rs[i], 16, t16))) break;
        const float ms = (t64 - t16) / 48.f;
        if (const char *vb = getenv("FDWAVE_TUNE_VERBOSE"))
            if (vb[0] == '1') fprintf(stderr, "fdwave batch tune: R %d: %.4f ms per step\n", rs[i], ms);
        if (ms < 0.98f * best) {
            best = ms;
            bestR = rs[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    std::lock_guard<std::mutex> lock(g_batch_mu);
    g_batch_tune[batch_key(nshots, shots)] = bestR;
    return FD_OK;
}

// ---------------------------- batched gradient ----------------------------
// The checkpointed adjoint gradient of many shots.  For 2D shots of a cross
// stencil with M = 2, 4 or 8 every step of each sweep (forward with
// checkpoints, segment recompute storing D, adjoint with the fused gradient)
// is one launch of the batched tile kernel over the tiles of every shot; each
// shot keeps its own buffers, checkpoints, segment and accumulator, so its
// gradient is bit for bit the one fd_adjoint_gradient gives.  Other batches
// run the shots one after another.

namespace {

std::vector<fd_shot> as_shots(int nshots, const fd_grad_shot *g)
{
    std::vector<fd_shot> v(nshots);
    for (int i = 0; i < nshots; ++i) {
        std::memset(&v[i], 0, sizeof v[i]);
        v[i].plan = g[i].plan;
        v[i].nsrc = g[i].nsrc;
        v[i].nrec = g[i].nrec;
    }
    return v;
}

size_t grad_batch_bytes(int nshots, const fd_grad_shot *shots, int k, bool one,
                        const std::vector<TileGeo> &geo, int64_t *ntiles_out)
{
    size_t tot = 0;
    int64_t ntiles = 0;
    for (int i = 0; i < nshots; ++i) {
        const fd_plan *p = shots[i].plan;
        const int kk = std::min(k, std::max(p->prob.nt, 1));
        tot += make_layout(p, shots[i].nsrc, shots[i].nrec, true, kk, one ? geo[i].ntiles : -1).total;
        if (one) ntiles += geo[i].ntiles;
    }
    if (one) tot += 2 * up(nshots * sizeof(ShotDesc)) + 3 * up(ntiles * sizeof(TileRec));
    if (ntiles_out) *ntiles_out = ntiles;
    return tot;
}

}  // namespace

extern "C" int fd_adjoint_gradient_batched_workspace_size(int nshots, const fd_grad_shot *shots,
                                                          int ckpt_every, size_t *bytes)
{
    clear_error();
    if (nshots < 0 || (nshots > 0 && !shots) || !bytes || ckpt_every < 1)
        return set_error(FD_ERR_ARG, "bad argument");
    for (int i = 0; i < nshots; ++i)
        if (!shots[i].plan) return set_error(FD_ERR_ARG, "shot %d has no plan", i);
    // enough for every tile shape the batch can take (the tuned one included)
    std::vector<fd_shot> fs = as_shots(nshots, shots);
    int rs[4] = {2};
    const int nr = nshots > 0 ? batch2d_variants(shots[0].plan->shape_eff, shots[0].plan->st.M, rs, 4) : 0;
    size_t tot = 0;
    for (int i = 0; i < std::max(nr, 1); ++i) {
        Variant bv;
        std::vector<TileGeo> geo;
        const bool one = nshots > 0 && batch_geometry(nshots, fs.data(), bv, geo, rs[i]);
        tot = std::max(tot, grad_batch_bytes(nshots, shots, ckpt_every, one, geo, nullptr));
    }
    *bytes = tot;
    return FD_OK;
}

extern "C" int fd_adjoint_gradient_batched(int nshots, const fd_grad_shot *shots, int k, void *ws,
                                           size_t ws_bytes, void *stream)
{
    clear_error();
    size_t need = 0;
    int st = fd_adjoint_gradient_batched_workspace_size(nshots, shots, k, &need);
    if (st) return st;
    if (!ws || ws_bytes < need) return set_error(FD_ERR_NOMEM, "workspace too small (%zu < %zu)", ws_bytes, need);
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return set_error(FD_ERR_ARG, "workspace must be 256-byte aligned");
    if (nshots == 0) return FD_OK;
    const fd_plan *p0 = shots[0].plan;
    for (int i = 1; i < nshots; ++i) {
        const fd_plan *q = shots[i].plan;
        if (q->prob.dim != p0->prob.dim || q->prob.nt != p0->prob.nt || q->prob.dt != p0->prob.dt ||
            q->st.M != p0->st.M || q->st.shape != p0->st.shape || q->st.scheme != p0->st.scheme ||
            std::memcmp(q->W, p0->W, sizeof q->W) != 0)
            return set_error(FD_ERR_ARG, "shot %d: batched shots must share dim, stencil, dt and nt", i);
    }
    for (int i = 0; i < nshots; ++i)
        if (!shots[i].grad_d || (shots[i].nrec > 0 && !shots[i].resid_d))
            return set_error(FD_ERR_ARG, "shot %d needs a gradient output and residuals", i);
    Variant bv;
    std::vector<TileGeo> geo;
    std::vector<fd_shot> fs = as_shots(nshots, shots);
    const bool one = batch_geometry(nshots, fs.data(), bv, geo);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *base = reinterpret_cast<char *>(ws);
    if (!one) {   // shot by shot, each in its slice of the workspace
        for (int i = 0; i < nshots; ++i) {
            const fd_grad_shot &g = shots[i];
            fd_plan *p = const_cast<fd_plan *>(g.plan);
            const int kk = std::min(k, std::max(p->prob.nt, 1));
            const size_t b = make_layout(p, g.nsrc, g.nrec, true, kk).total;
            st = fd_adjoint_gradient(p, g.model_kind, g.model_d, g.nsrc, g.src_idx, g.wavelet_d, g.nrec,
                                     g.rec_idx, g.resid_d, k, g.grad_d, g.traces_d, nullptr, base, b, stream);
            if (st) return set_error(st, "shot %d: %s", i, fd_last_error());
            base += b;
        }
        return FD_OK;
    }
    const int nt = p0->prob.nt;
    k = std::min(k, std::max(nt, 1));
    const int nck = (nt + k - 1) / k;
    int64_t ntiles_all = 0;
    size_t shots_bytes = 0;
    for (int i = 0; i < nshots; ++i) {
        shots_bytes += make_layout(shots[i].plan, shots[i].nsrc, shots[i].nrec, true, k, geo[i].ntiles).total;
        ntiles_all += geo[i].ntiles;
    }
    char *xd = base + shots_bytes;                      // forward descriptors
    char *xa = xd + up(nshots * sizeof(ShotDesc));      // adjoint descriptors
    char *xr = xa + up(nshots * sizeof(ShotDesc));      // tile records: forward | recompute | adjoint
    const size_t rb = up(ntiles_all * sizeof(TileRec));
    std::vector<ShotDesc> df(nshots), da(nshots);
    std::vector<TileRec> rf, rr, ra;
    struct ShotBufs {
        float *buf[4];
        char *ckpt;
        float *gacc;
        size_t fb;
    };
    std::vector<ShotBufs> sb(nshots);
    for (int i = 0; i < nshots; ++i) {
        fd_plan *p = const_cast<fd_plan *>(shots[i].plan);
        const fd_grad_shot &g = shots[i];
        const Layout L = make_layout(p, g.nsrc, g.nrec, true, k, geo[i].ntiles);
        st = check_common(p, g.model_kind, g.model_d, g.nsrc, g.src_idx, g.wavelet_d, g.nrec, g.rec_idx,
                          base, L.total, L.total);
        if (st) return set_error(st, "shot %d: %s", i, fd_last_error());
        if ((st = ensure_tuned(p))) return st;
        Tables T;
        if ((st = make_tables(p, g.nsrc, g.src_idx, g.nrec, g.rec_idx, true, T, &geo[i]))) return st;
        if ((st = upload_tables(p, L, base, T, s))) return st;
        FDW_CK(cudaMemsetAsync(base + L.status, 0, kAlign, s));
        const size_t fb = up((size_t)p->field * sizeof(float));
        ShotBufs &b = sb[i];
        b.fb = fb;
        for (int j = 0; j < 4; ++j) {
            b.buf[j] = reinterpret_cast<float *>(base + L.buf[j]);
            FDW_CK(cudaMemsetAsync(b.buf[j], 0, fb, s));
        }
        b.gacc = reinterpret_cast<float *>(base + L.gacc);
        FDW_CK(cudaMemsetAsync(b.gacc, 0, fb, s));
        b.ckpt = base + L.ckpt;
        if ((st = prep_model(p, L, base, g.model_kind, g.model_d, s))) return st;
        const float *kap = reinterpret_cast<const float *>(base + L.kappa);
        float *dseg = reinterpret_cast<float *>(base + L.dseg);
        auto fill = [&](ShotDesc &d, float *b0, float *b1) -> int {
            std::memset(&d, 0, sizeof d);
            Variant keep = p->var;
            p->var = bv;
            int r = encode_field_map(p, &d.tmap[0], b0, false);
            r = r ? r : encode_field_map(p, &d.tmap[1], b1, false);
            r = r ? r : encode_field_map(p, &d.tile[0], b0, true);
            r = r ? r : encode_field_map(p, &d.tile[1], b1, true);
            r = r ? r : encode_field_map(p, &d.ktile, kap, true);
            p->var = keep;
            d.info.buf[0] = b0;
            d.info.buf[1] = b1;
            d.info.kappa = kap;
            d.info.nx = p->pad[2];
            d.info.nz = p->pad[0];
            d.info.pitch = p->pitch;
            d.info.phys_lo[0] = p->prob.nb; d.info.phys_hi[0] = p->prob.nb + p->prob.n[2] - 1;
            d.info.phys_lo[2] = p->prob.nb; d.info.phys_hi[2] = p->prob.nb + p->prob.n[0] - 1;
            d.info.gcoef = p->gcoef;
            d.info.tiles_x = geo[i].tiles_x;
            d.info.dseg = dseg;
            d.info.field = (int64_t)(fb / sizeof(float));
            return r;
        };
        if (fill(df[i], b.buf[0], b.buf[1]) || fill(da[i], b.buf[2], b.buf[3]))
            return set_error(FD_ERR_CUDA, "cuTensorMapEncodeTiled failed");
        // forward / recompute: sources in, receivers out; adjoint: residuals in
        df[i].info.inj = reinterpret_cast<const PtEntry *>(base + L.tab + T.inj);
        df[i].info.inj_series = g.wavelet_d;
        df[i].info.inj_ncol = g.nsrc;
        df[i].info.smp = reinterpret_cast<const PtEntry *>(base + L.tab + T.smp);
        df[i].info.smp_out = g.traces_d;
        df[i].info.smp_ncol = g.nrec;
        da[i].info.inj = reinterpret_cast<const PtEntry *>(base + L.tab + T.ainj);
        da[i].info.inj_series = g.resid_d;
        da[i].info.inj_ncol = g.nrec;
        da[i].info.gacc = b.gacc;
        const int32_t *hip = reinterpret_cast<const int32_t *>(T.blob.data() + T.inj_ptr);
        const int32_t *hsp = reinterpret_cast<const int32_t *>(T.blob.data() + T.smp_ptr);
        const int32_t *hap = reinterpret_cast<const int32_t *>(T.blob.data() + T.ainj_ptr);
        for (int t = 0; t < geo[i].ntiles; ++t) {
            TileRec r;
            std::memset(&r, 0, sizeof r);
            r.shot = i;
            r.tile = t;
            r.x0 = (t % geo[i].tiles_x) * geo[i].tx;
            r.z0 = (t / geo[i].tiles_x) * geo[i].tz;
            TileRec a = r;
            r.ib = g.nsrc ? hip[t] : 0;
            r.ie = g.nsrc ? hip[t + 1] : 0;
            TileRec c = r;            // recompute: no sampling
            r.sb = (g.nrec && g.traces_d) ? hsp[t] : 0;
            r.se = (g.nrec && g.traces_d) ? hsp[t + 1] : 0;
            a.ib = g.nrec ? hap[t] : 0;
            a.ie = g.nrec ? hap[t + 1] : 0;
            rf.push_back(r);
            rr.push_back(c);
            ra.push_back(a);
        }
        base += L.total;
    }
    FDW_CK(cudaMemcpyAsync(xd, df.data(), nshots * sizeof(ShotDesc), cudaMemcpyHostToDevice, s));
    FDW_CK(cudaMemcpyAsync(xa, da.data(), nshots * sizeof(ShotDesc), cudaMemcpyHostToDevice, s));
    FDW_CK(cudaMemcpyAsync(xr, rf.data(), ntiles_all * sizeof(TileRec), cudaMemcpyHostToDevice, s));
    FDW_CK(cudaMemcpyAsync(xr + rb, rr.data(), ntiles_all * sizeof(TileRec), cudaMemcpyHostToDevice, s));
    FDW_CK(cudaMemcpyAsync(xr + 2 * rb, ra.data(), ntiles_all * sizeof(TileRec), cudaMemcpyHostToDevice, s));
    BatchParams bp;
    std::memset(&bp, 0, sizeof bp);
    bp.ntiles = (int)ntiles_all;
    bp.status = reinterpret_cast<int *>(ws);     // shot 0's status word
    std::memcpy(bp.w, p0->W, sizeof bp.w);
    const ShotDesc *dfd = reinterpret_cast<const ShotDesc *>(xd);
    const ShotDesc *dad = reinterpret_cast<const ShotDesc *>(xa);
    const TileRec *trf = reinterpret_cast<const TileRec *>(xr);
    const TileRec *trr = reinterpret_cast<const TileRec *>(xr + rb);
    const TileRec *tra = reinterpret_cast<const TileRec *>(xr + 2 * rb);
    // forward sweep with checkpoints (u^n, u^{n-1}) at n = c k; with one
    // segment (k >= nt) it stores D of every step instead, as in
    // fd_adjoint_gradient, and the backward sweep recomputes nothing
    const bool store_all = nck == 1;
    bp.shots = dfd;
    bp.tiles = trf;
    for (int n = 0; n < nt; ++n) {
        const int cur = n & 1;
        if (n % k == 0 && !store_all)
            for (int i = 0; i < nshots; ++i) {
                const int c = n / k;
                FDW_CK(cudaMemcpyAsync(sb[i].ckpt + (size_t)(2 * c) * sb[i].fb, sb[i].buf[cur], sb[i].fb,
                                       cudaMemcpyDeviceToDevice, s));
                FDW_CK(cudaMemcpyAsync(sb[i].ckpt + (size_t)(2 * c + 1) * sb[i].fb, sb[i].buf[cur ^ 1],
                                       sb[i].fb, cudaMemcpyDeviceToDevice, s));
            }
        bp.step = n;
        bp.parity = cur;
        bp.seg = store_all ? n : 0;
        bp.check = check_step(n, nt);
        FDW_CK(launch_batched2d(bv, bp, (int)ntiles_all, s, store_all ? kModeStoreD : kModeForward));
    }
    // backward sweep over segments: restore, recompute storing D, adjoint steps
    int t = 0;
    for (int c = nck - 1; c >= 0; --c) {
        const int k0 = c * k, k1 = std::min(k0 + k, nt);
        if (!store_all) {
            for (int i = 0; i < nshots; ++i) {
                FDW_CK(cudaMemcpyAsync(sb[i].buf[0], sb[i].ckpt + (size_t)(2 * c) * sb[i].fb, sb[i].fb,
                                       cudaMemcpyDeviceToDevice, s));
                FDW_CK(cudaMemcpyAsync(sb[i].buf[1], sb[i].ckpt + (size_t)(2 * c + 1) * sb[i].fb, sb[i].fb,
                                       cudaMemcpyDeviceToDevice, s));
            }
            bp.shots = dfd;
            bp.tiles = trr;
            bp.check = 0;   // the recompute repeats the checked forward sweep bit for bit
            for (int n = k0; n < k1; ++n) {
                bp.step = n;
                bp.parity = (n - k0) & 1;
                bp.seg = n - k0;
                FDW_CK(launch_batched2d(bv, bp, (int)ntiles_all, s, kModeStoreD));
            }
        }
        bp.shots = dad;
        bp.tiles = tra;
        for (int j = k1; j > k0; --j, ++t) {
            bp.step = j - 1;
            bp.parity = t & 1;
            bp.seg = j - 1 - k0;
            bp.check = check_step(t, nt);
            FDW_CK(launch_batched2d(bv, bp, (int)ntiles_all, s, kModeAdjoint));
        }
    }
    for (int i = 0; i < nshots; ++i) {
        const fd_plan *p = shots[i].plan;
        const fd_problem &pr = p->prob;
        const int64_t phys[3] = {pr.n[0], pr.n[1], pr.n[2]};
        FDW_CK(launch_fold_grad(sb[i].gacc, p->pitch, zstride(p), phys, pr.nb, (float)(-1.0 / (pr.dt * pr.dt)),
                                shots[i].grad_d, s));
    }
    return FD_OK;
}
