// Evaluation metrics of the paper on the GPU, in FP64 arithmetic on FP32 data:
// the classical error norms of Section 2.4 (Eqs. snapnorm1, snapnorm2,
// snapnormmax), the DFT-based dispersion metric of Appendix A (Eqs. dft,
// ampldft, phasedft, phasesdifdft, phasesdifdftajusted, gammadft,
// norm2gammastdft, norm2gammarecdftavg, norm2gammarecdftmax) and its wavelet
// counterpart (Eqs. omegak, cwt1, cwt2, cwt3, cwt, amplcwt, phasecwt,
// amplmaxcwt, phasesdifcwt, phasesdifcwtajusted, gammacwt, norm2gammastcwt,
// norm2gammareccwtavg, norm2gammareccwtmax).
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "runtime.h"

namespace fdw {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kPiM14 = 0.75112554446494248286;   // pi^(-1/4)

// A[p][k] = sum_n u[n][p] exp(-2 pi i k n / nt) for receiver p (thread x) and
// frequency k (thread y); u is [nt][nrec] (receivers contiguous, as the
// traces of fd_forward).  The twiddle advances by a complex rotation and is
// re-seeded from the exact angle every 64 samples.
__global__ void dft_kernel(const float *__restrict__ u, int nt, int nrec, int nfreq,
                           double2 *__restrict__ A)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y * blockDim.y + threadIdx.y;
    if (p >= nrec || k >= nfreq) return;
    double ws, wc;
    sincospi(-2.0 * (double)k / (double)nt, &ws, &wc);
    double zs = 0.0, zc = 1.0, re = 0.0, im = 0.0;
    for (int n = 0; n < nt; ++n) {
        if ((n & 63) == 0) {
            const long long m = ((long long)k * n) % nt;
            sincospi(-2.0 * (double)m / (double)nt, &zs, &zc);
        }
        const double v = u[(long long)n * nrec + p];
        re = fma(v, zc, re);
        im = fma(v, zs, im);
        const double c = zc * wc - zs * ws;
        zs = zc * ws + zs * wc;
        zc = c;
    }
    A[(long long)p * nfreq + k] = make_double2(re, im);
}

template <bool MAX>
__device__ double block_reduce(double v, double *red)
{
    const int t = threadIdx.x;
    red[t] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (t < s) red[t] = MAX ? fmax(red[t], red[t + s]) : red[t] + red[t + s];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// One block per receiver: gamma_k = (wrapped phase difference / pi) *
// (|A_k^num| / max_k |A_k^num|) and the trace norm sqrt(mean_k gamma_k^2).
__global__ void gamma_kernel(const double2 *__restrict__ An, const double2 *__restrict__ Ar,
                             int nfreq, float *gamma, double *norm)
{
    __shared__ double red[256];
    const int p = blockIdx.x;
    const double2 *a = An + (long long)p * nfreq, *b = Ar + (long long)p * nfreq;
    double mx = 0.0;
    for (int k = threadIdx.x; k < nfreq; k += blockDim.x) mx = fmax(mx, hypot(a[k].x, a[k].y));
    const double amax = block_reduce<true>(mx, red);
    double s = 0.0;
    for (int k = threadIdx.x; k < nfreq; k += blockDim.x) {
        double d = atan2(a[k].y, a[k].x) - atan2(b[k].y, b[k].x);
        if (d > kPi) d -= 2.0 * kPi;
        else if (d < -kPi) d += 2.0 * kPi;
        const double g = amax > 0.0 ? (d / kPi) * (hypot(a[k].x, a[k].y) / amax) : 0.0;
        if (gamma) gamma[(long long)p * nfreq + k] = (float)g;
        s += g * g;
    }
    const double tot = block_reduce<false>(s, red);
    if (threadIdx.x == 0) norm[p] = sqrt(tot / nfreq);
}

// agg = (average, maximum) of the trace norms.
__global__ void aggregate_kernel(const double *norm, int nrec, double *agg)
{
    __shared__ double red[256];
    double s = 0.0, m = 0.0;
    for (int p = threadIdx.x; p < nrec; p += blockDim.x) {
        s += norm[p];
        m = fmax(m, norm[p]);
    }
    const double ts = block_reduce<false>(s, red);
    const double tm = block_reduce<true>(m, red);
    if (threadIdx.x == 0) {
        agg[0] = ts / nrec;
        agg[1] = tm;
    }
}

// Morlet CWT of one trace at one scale (block (k, p, signal)):
// S_{n,k} = (1/nt) sum_{k'=1}^{nt/2} A_k' Psi(s_k omega_k') exp(+2 pi i k' n / nt),
// Psi(s omega) = (2 pi s / tau)^(1/2) pi^(-1/4) exp(-(s omega - omega0)^2 / 2) for
// omega > 0, with s_k omega_k' = c k'/k and 2 pi s_k / tau = c nt / k.  The
// weighted lines B_k' are staged in shared memory; each thread sums them for
// its times n with a twiddle that advances by a complex rotation and is
// re-seeded from the exact angle every 64 lines.  Scale 0 is zero.
__global__ void cwt_kernel(const double2 *__restrict__ An, const double2 *__restrict__ Ar,
                           int nt, int nh, int nscale, double c, double omega0,
                           double2 *__restrict__ Sn, double2 *__restrict__ Sr)
{
    extern __shared__ double2 B[];
    const int k = blockIdx.x, p = blockIdx.y;
    const double2 *A = (blockIdx.z ? Ar : An) + (long long)p * nh;
    double2 *S = (blockIdx.z ? Sr : Sn) + ((long long)p * nscale + k) * nt;
    if (k == 0) {
        for (int n = threadIdx.x; n < nt; n += blockDim.x) S[n] = make_double2(0.0, 0.0);
        return;
    }
    const double scale = sqrt(c * (double)nt / (double)k) * kPiM14 / (double)nt;
    for (int j = threadIdx.x; j < nh; j += blockDim.x) {
        double2 b = make_double2(0.0, 0.0);
        if (j >= 1 && 2 * j <= nt) {
            const double x = c * (double)j / (double)k - omega0;
            const double g = scale * exp(-0.5 * x * x);
            b = make_double2(A[j].x * g, A[j].y * g);
        }
        B[j] = b;
    }
    __syncthreads();
    for (int n = threadIdx.x; n < nt; n += blockDim.x) {
        double ws, wc, zs = 0.0, zc = 1.0, re = 0.0, im = 0.0;
        sincospi(2.0 * (double)n / (double)nt, &ws, &wc);
        for (int j = 1; j < nh; ++j) {
            if (((j - 1) & 63) == 0) {
                const long long m = ((long long)j * n) % nt;
                sincospi(2.0 * (double)m / (double)nt, &zs, &zc);
            }
            const double2 b = B[j];
            re = fma(b.x, zc, fma(-b.y, zs, re));
            im = fma(b.x, zs, fma(b.y, zc, im));
            const double t = zc * wc - zs * ws;
            zs = zc * ws + zs * wc;
            zc = t;
        }
        S[n] = make_double2(re, im);
    }
}

// amax[p] = max over (k, n) of |S^num_{n,k}| (amax starts at zero; non-negative
// doubles compare like their bit patterns).
__global__ void amp_max_kernel(const double2 *__restrict__ S, long long per, double *amax)
{
    __shared__ double red[256];
    const int p = blockIdx.y;
    const double2 *s = S + (long long)p * per;
    double m = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < per;
         i += (long long)gridDim.x * blockDim.x)
        m = fmax(m, hypot(s[i].x, s[i].y));
    m = block_reduce<true>(m, red);
    if (threadIdx.x == 0)
        atomicMax(reinterpret_cast<unsigned long long *>(&amax[p]),
                  (unsigned long long)__double_as_longlong(m));
}

// gamma_{n,k} for scale k of receiver p (block (k, p)); sumsq[p] accumulates
// gamma^2 (starts at zero).
__global__ void gamma_w_kernel(const double2 *__restrict__ Sn, const double2 *__restrict__ Sr,
                               int nt, int nscale, const double *amax, float *gamma,
                               double *sumsq)
{
    __shared__ double red[256];
    const int k = blockIdx.x, p = blockIdx.y;
    const long long o = ((long long)p * nscale + k) * nt;
    const double am = amax[p];
    double s = 0.0;
    for (int n = threadIdx.x; n < nt; n += blockDim.x) {
        const double2 a = Sn[o + n], b = Sr[o + n];
        double d = atan2(a.y, a.x) - atan2(b.y, b.x);
        if (d > kPi) d -= 2.0 * kPi;
        else if (d < -kPi) d += 2.0 * kPi;
        const double g = am > 0.0 ? (d / kPi) * (hypot(a.x, a.y) / am) : 0.0;
        if (gamma) gamma[o + n] = (float)g;
        s += g * g;
    }
    s = block_reduce<false>(s, red);
    if (threadIdx.x == 0) atomicAdd(&sumsq[p], s);
}

__global__ void mean_sqrt_kernel(double *v, int n, double count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = sqrt(v[i] / count);
}

// acc = (sum |a - b|, sum (a - b)^2, max |a - b|); acc starts at zero.  The
// maximum of non-negative doubles is the maximum of their bit patterns.
__global__ void norms_kernel(const float *__restrict__ a, const float *__restrict__ b,
                             long long n, double *acc)
{
    __shared__ double red[256];
    double s1 = 0.0, s2 = 0.0, mx = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double d = fabs((double)a[i] - (double)b[i]);
        s1 += d;
        s2 = fma(d, d, s2);
        mx = fmax(mx, d);
    }
    s1 = block_reduce<false>(s1, red);
    s2 = block_reduce<false>(s2, red);
    mx = block_reduce<true>(mx, red);
    if (threadIdx.x == 0) {
        atomicAdd(&acc[0], s1);
        atomicAdd(&acc[1], s2);
        atomicMax(reinterpret_cast<unsigned long long *>(&acc[2]),
                  (unsigned long long)__double_as_longlong(mx));
    }
}

__global__ void norms_finish(double *acc, double scale1, double scale2)
{
    acc[0] *= scale1;
    acc[1] = scale2 * sqrt(acc[1]);
}

}  // namespace

}  // namespace fdw

using namespace fdw;

extern "C" int fd_error_norms(const float *num_d, const float *ref_d, int64_t n, double scale1,
                              double scale2, double *out_d, void *stream)
{
    clear_error();
    if (n < 0 || !out_d || (n > 0 && (!num_d || !ref_d))) return set_error(FD_ERR_ARG, "bad argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(out_d, 0, 3 * sizeof(double), s) != cudaSuccess)
        return set_error(FD_ERR_CUDA, "cudaMemsetAsync failed");
    if (n > 0) {
        const long long blocks = std::min<long long>((n + 255) / 256, 152 * 8);
        norms_kernel<<<(int)blocks, 256, 0, s>>>(num_d, ref_d, n, out_d);
    }
    norms_finish<<<1, 1, 0, s>>>(out_d, scale1, scale2);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FD_OK : set_error(FD_ERR_CUDA, "%s", cudaGetErrorString(e));
}

extern "C" int fd_dft_gamma(const float *num_d, const float *ref_d, int nt, int nrec, int nfreq,
                            double *spec_num_d, double *spec_ref_d, float *gamma_d,
                            double *norm_d, double *agg_d, void *stream)
{
    clear_error();
    if (nt <= 0 || nrec <= 0 || nfreq <= 0 || nfreq > nt || !num_d || !ref_d || !spec_num_d ||
        !spec_ref_d || !norm_d)
        return set_error(FD_ERR_ARG, "bad argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const dim3 blk(32, 8), grd((nrec + 31) / 32, (nfreq + 7) / 8);
    double2 *An = reinterpret_cast<double2 *>(spec_num_d), *Ar = reinterpret_cast<double2 *>(spec_ref_d);
    dft_kernel<<<grd, blk, 0, s>>>(num_d, nt, nrec, nfreq, An);
    dft_kernel<<<grd, blk, 0, s>>>(ref_d, nt, nrec, nfreq, Ar);
    gamma_kernel<<<nrec, 256, 0, s>>>(An, Ar, nfreq, gamma_d, norm_d);
    if (agg_d) aggregate_kernel<<<1, 256, 0, s>>>(norm_d, nrec, agg_d);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FD_OK : set_error(FD_ERR_CUDA, "%s", cudaGetErrorString(e));
}

extern "C" int fd_cwt_gamma(const float *num_d, const float *ref_d, int nt, int nrec, int nscale,
                            double omega0, double *spec_num_d, double *spec_ref_d,
                            double *cwt_num_d, double *cwt_ref_d, float *gamma_d, double *amax_d,
                            double *norm_d, double *agg_d, void *stream)
{
    clear_error();
    if (nt <= 0 || nrec <= 0 || nrec > 65535 || nscale <= 0 || nscale > nt || !(omega0 > 0.0) || !num_d ||
        !ref_d || !spec_num_d || !spec_ref_d || !cwt_num_d || !cwt_ref_d || !amax_d || !norm_d)
        return set_error(FD_ERR_ARG, "bad argument");
    const int nh = nt / 2 + 1;
    const size_t smem = (size_t)nh * sizeof(double2);
    if (smem > 227u * 1024u)
        return set_error(FD_ERR_ARG, "nt = %d: the DFT lines of a trace exceed shared memory "
                         "(nt <= 29054)", nt);
    if (smem > 48u * 1024u &&
        cudaFuncSetAttribute(cwt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return set_error(FD_ERR_CUDA, "cudaFuncSetAttribute failed");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    double2 *An = reinterpret_cast<double2 *>(spec_num_d), *Ar = reinterpret_cast<double2 *>(spec_ref_d);
    double2 *Sn = reinterpret_cast<double2 *>(cwt_num_d), *Sr = reinterpret_cast<double2 *>(cwt_ref_d);
    if (cudaMemsetAsync(amax_d, 0, nrec * sizeof(double), s) != cudaSuccess ||
        cudaMemsetAsync(norm_d, 0, nrec * sizeof(double), s) != cudaSuccess)
        return set_error(FD_ERR_CUDA, "cudaMemsetAsync failed");
    const dim3 blk(32, 8), grd((nrec + 31) / 32, (nh + 7) / 8);
    dft_kernel<<<grd, blk, 0, s>>>(num_d, nt, nrec, nh, An);
    dft_kernel<<<grd, blk, 0, s>>>(ref_d, nt, nrec, nh, Ar);
    const double c = 0.5 * (omega0 + std::sqrt(2.0 + omega0 * omega0));
    cwt_kernel<<<dim3(nscale, nrec, 2), 256, smem, s>>>(An, Ar, nt, nh, nscale, c, omega0, Sn, Sr);
    const long long per = (long long)nscale * nt;
    const int chunks = (int)std::min<long long>((per + 255) / 256, 1024);
    amp_max_kernel<<<dim3(chunks, nrec), 256, 0, s>>>(Sn, per, amax_d);
    gamma_w_kernel<<<dim3(nscale, nrec), 256, 0, s>>>(Sn, Sr, nt, nscale, amax_d, gamma_d, norm_d);
    mean_sqrt_kernel<<<(nrec + 255) / 256, 256, 0, s>>>(norm_d, nrec, (double)per);
    if (agg_d) aggregate_kernel<<<1, 256, 0, s>>>(norm_d, nrec, agg_d);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FD_OK : set_error(FD_ERR_CUDA, "%s", cudaGetErrorString(e));
}
