// Auxiliary kernels: padded coefficient field from the model, state copies
// between the pitched field buffers and packed arrays, gradient fold, and the
// tensor-map encoder (driver entry point resolved at run time).
#include <cudaTypedefs.h>

#include "device_common.cuh"

namespace fdw {

namespace {

// kappa = (v dt / h)^2 on the padded grid; the physical model is extended
// into the sponge by edge replication.  Pitch columns beyond nx get 0.
__global__ void prep_kappa_kernel(const float *__restrict__ model, int kind, float *kappa,
                                  int64_t pz, int64_t py, int64_t px, int64_t nz, int64_t ny,
                                  int64_t nx, int nb, int64_t pitch, int64_t plane,
                                  double c2, float vmax2, int *status)
{
    const int64_t total = pz * py * pitch;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = i % pitch, r = i / pitch, y = r % py, z = r / py;
        float out = 0.f;
        if (x < px) {
            const int64_t iz = min(max(z - nb, (int64_t)0), nz - 1);
            const int64_t iy = min(max(y - (py > 1 ? nb : 0), (int64_t)0), ny - 1);
            const int64_t ix = min(max(x - nb, (int64_t)0), nx - 1);
            const float m = model[(iz * ny + iy) * nx + ix];
            const float v2 = kind == FD_MODEL_VELOCITY ? m * m : 1.0f / m;
            if (!(v2 <= vmax2)) atomicOr(status, kStatusVmax);
            out = static_cast<float>(c2 * static_cast<double>(v2));
        }
        kappa[z * plane + y * pitch + x] = out;
    }
}

__global__ void copy_state_kernel(const float *__restrict__ src, int64_t sp, int64_t spl,
                                  float *dst, int64_t dp, int64_t dpl, int64_t pz, int64_t py,
                                  int64_t px)
{
    const int64_t total = pz * py * px;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = i % px, r = i / px, y = r % py, z = r / py;
        dst[z * dpl + y * dp + x] = src[z * spl + y * sp + x];
    }
}

// grad[phys] = scale * sum of gacc over the padded nodes that replicate it.
__global__ void fold_grad_kernel(const float *__restrict__ g, int64_t pitch, int64_t plane,
                                 int64_t nz, int64_t ny, int64_t nx, int nb, int ydim,
                                 float scale, float *grad)
{
    const int64_t total = nz * ny * nx;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ix = i % nx, r = i / nx, iy = r % ny, iz = r / ny;
        auto range = [nb](int64_t k, int64_t n, int64_t &lo, int64_t &hi) {
            lo = k == 0 ? 0 : k + nb;
            hi = k == n - 1 ? n - 1 + 2 * nb : k + nb;
        };
        int64_t z0, z1, y0, y1, x0, x1;
        range(iz, nz, z0, z1);
        range(ix, nx, x0, x1);
        if (ydim) range(iy, ny, y0, y1);
        else y0 = y1 = 0;
        double s = 0.0;
        for (int64_t z = z0; z <= z1; ++z)
            for (int64_t y = y0; y <= y1; ++y)
                for (int64_t x = x0; x <= x1; ++x) s += g[z * plane + y * pitch + x];
        grad[i] = static_cast<float>(scale * s);
    }
}

int grid_for(int64_t n)
{
    int64_t b = (n + 255) / 256;
    return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

}  // namespace

cudaError_t launch_prep_kappa(const float *model, int kind, float *kappa, int dim,
                              const int64_t phys[3], int nb, const int64_t pad[3],
                              int64_t pitch, int64_t plane, double dt_over_h,
                              float vmax_sq_limit, int *status, cudaStream_t s)
{
    const int64_t total = pad[0] * pad[1] * pitch;
    prep_kappa_kernel<<<grid_for(total), 256, 0, s>>>(
        model, kind, kappa, pad[0], pad[1], pad[2], phys[0], phys[1], phys[2], nb, pitch, plane,
        dt_over_h * dt_over_h, vmax_sq_limit, status);
    (void)dim;
    return cudaGetLastError();
}

cudaError_t launch_copy_state(const float *src, int64_t src_pitch, int64_t src_plane,
                              float *dst, int64_t dst_pitch, int64_t dst_plane,
                              const int64_t pad[3], cudaStream_t s)
{
    const int64_t total = pad[0] * pad[1] * pad[2];
    copy_state_kernel<<<grid_for(total), 256, 0, s>>>(src, src_pitch, src_plane, dst, dst_pitch,
                                                       dst_plane, pad[0], pad[1], pad[2]);
    return cudaGetLastError();
}

cudaError_t launch_fold_grad(const float *gacc, int64_t pitch, int64_t plane,
                             const int64_t phys[3], int nb, float scale, float *grad,
                             cudaStream_t s)
{
    const int64_t total = phys[0] * phys[1] * phys[2];
    fold_grad_kernel<<<grid_for(total), 256, 0, s>>>(gacc, pitch, plane, phys[0], phys[1],
                                                     phys[2], nb, phys[1] > 1 ? 1 : 0, scale,
                                                     grad);
    return cudaGetLastError();
}

int encode_tmap(CUtensorMap *map, const float *base, int rank, const int64_t *dims,
                const int64_t *strides_bytes, const int *box)
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p)
            return -1;
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    cuuint64_t gdim[3], gstr[2];
    cuuint32_t bdim[3], estr[3] = {1, 1, 1};
    for (int i = 0; i < rank; ++i) {
        gdim[i] = (cuuint64_t)dims[i];
        bdim[i] = (cuuint32_t)box[i];
    }
    for (int i = 0; i + 1 < rank; ++i) gstr[i] = (cuuint64_t)strides_bytes[i];
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank,
                    const_cast<float *>(base), gdim, gstr, bdim, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : (int)r;
}

}  // namespace fdw
