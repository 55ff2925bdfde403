// HEALPix maps of per-ray quantities (Sect. 2.4) and the deflection angle alpha = theta - beta.
//
// Rays shot at pixel centres give maps directly (ray i = pixel i); rays at other directions (a
// finer resolution, a geodesic finder's solutions) are binned: each direction is assigned its
// HEALPix pixel (Gorski et al. 2005: z = cos theta and the quarter coordinate t = phi / (pi/2);
// edge-line indices in the equatorial zone |z| <= 2/3, polar-cap indices from sqrt(3 (1 - |z|))),
// and every quantity is added into its pixel with an FP64 atomic.  mean = sums / counts.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "mt_trace_device.cuh"

namespace mt {
namespace {

// Spread the low 32 bits of v to the even bit positions.
__device__ __forceinline__ unsigned long long spread2(unsigned long long v) {
  v &= 0xffffffffull;
  v = (v | (v << 16)) & 0x0000ffff0000ffffull;
  v = (v | (v << 8)) & 0x00ff00ff00ff00ffull;
  v = (v | (v << 4)) & 0x0f0f0f0f0f0f0f0full;
  v = (v | (v << 2)) & 0x3333333333333333ull;
  v = (v | (v << 1)) & 0x5555555555555555ull;
  return v;
}

__device__ long long healpix_of(long long N, double x, double y, double zc, bool nest) {
  const double r = sqrt(x * x + y * y + zc * zc);
  const double z = zc / r, za = fabs(z);
  double t = atan2(y, x) * (2.0 / 3.14159265358979323846);  // phi / (pi / 2)
  if (t < 0.0) t += 4.0;
  if (t >= 4.0) t -= 4.0;
  const long long npix = 12 * N * N;
  long long face, ix, iy;
  if (za <= 2.0 / 3.0) {
    const double u = N * (0.5 + t), w = 0.75 * N * z;
    const long long jp = (long long)floor(u - w);  // ascending edge line
    const long long jm = (long long)floor(u + w);  // descending edge line
    if (!nest) {
      const long long ring = N + 1 + jp - jm;  // 1 .. 2N + 1 counted from z = 2/3
      long long ip = (jp + jm - N + (1 - (ring & 1)) + 1) / 2;
      ip %= 4 * N;
      if (ip < 0) ip += 4 * N;
      return 2 * N * (N - 1) + (ring - 1) * 4 * N + ip;
    }
    const long long fp = jp / N, fm = jm / N;
    face = fp == fm ? (fp | 4) : (fp < fm ? fp : fm + 8);
    ix = jm & (N - 1);
    iy = N - (jp & (N - 1)) - 1;
  } else {
    long long q = (long long)t;
    if (q > 3) q = 3;
    const double tp = t - (double)q;
    const double s = N * sqrt(3.0 * (1.0 - za));
    long long jp = (long long)(tp * s), jm = (long long)((1.0 - tp) * s);
    if (!nest) {
      const long long ring = jp + jm + 1;  // counted from the nearer pole
      long long ip = (long long)(t * ring);
      ip %= 4 * ring;
      if (ip < 0) ip += 4 * ring;
      return z > 0.0 ? 2 * ring * (ring - 1) + ip : npix - 2 * ring * (ring + 1) + ip;
    }
    if (jp > N - 1) jp = N - 1;
    if (jm > N - 1) jm = N - 1;
    if (z > 0.0) {
      face = q;
      ix = N - jm - 1;
      iy = N - jp - 1;
    } else {
      face = q + 8;
      ix = jp;
      iy = jm;
    }
  }
  return face * N * N + (long long)(spread2((unsigned long long)ix) | (spread2((unsigned long long)iy) << 1));
}

__global__ void bin_kernel(const double* __restrict__ dirs, long long n, const double* __restrict__ values, int k,
                           long long nside, int nest, double* sums, double* counts, long long* ipix) {
  const long long npix = 12 * nside * nside;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long p = healpix_of(nside, dirs[i], dirs[n + i], dirs[2 * n + i], nest != 0);
    if (ipix) ipix[i] = p;
    if (counts) atomicAdd(&counts[p], 1.0);
    for (int q = 0; q < k; ++q) atomicAdd(&sums[(long long)q * npix + p], values[(long long)q * n + i]);
  }
}

__global__ void deflection_kernel(DevCones C, const double* __restrict__ dirs, const double* __restrict__ xi,
                                  long long n, double* alpha) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    int c = 0;
    while (c + 1 < C.n && C.begin[c + 1] <= i) ++c;
    double th[3] = {dirs[i], dirs[n + i], dirs[2 * n + i]};
    double be[3] = {xi[i] - C.obs[c][0], xi[n + i] - C.obs[c][1], xi[2 * n + i] - C.obs[c][2]};
    const double nt = sqrt(th[0] * th[0] + th[1] * th[1] + th[2] * th[2]);
    const double nb = sqrt(be[0] * be[0] + be[1] * be[1] + be[2] * be[2]);
    double d[3];
    for (int q = 0; q < 3; ++q) {
      th[q] /= nt;
      be[q] /= nb;
      d[q] = th[q] - be[q];
    }
    double e1[3], e2[3];
    screen_vectors(th, e1, e2);
    const double cr[3] = {th[1] * be[2] - th[2] * be[1], th[2] * be[0] - th[0] * be[2], th[0] * be[1] - th[1] * be[0]};
    alpha[i] = d[0] * e1[0] + d[1] * e1[1] + d[2] * e1[2];
    alpha[n + i] = d[0] * e2[0] + d[1] * e2[1] + d[2] * e2[2];
    alpha[2 * n + i] = atan2(sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]),
                             th[0] * be[0] + th[1] * be[1] + th[2] * be[2]);
  }
}

int grid_for(long long n) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long blocks = (n + 255) / 256;
  const long long cap = (long long)sms * 8;
  return (int)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

}  // namespace
}  // namespace mt

using namespace mt;

extern "C" mt_status mt_healpix_bin(const double* dirs, int64_t n, const double* values, int32_t k, int64_t nside,
                                    int32_t nest, double* sums, double* counts, int64_t* ipix, void* stream) {
  if (n < 0 || k < 0 || nside < 1 || nside > (1ll << 28) || (nside & (nside - 1)) != 0) return MT_ERR_INVALID_ARG;
  if (nest != 0 && nest != 1) return MT_ERR_INVALID_ARG;
  if (n > 0 && !dirs) return MT_ERR_INVALID_ARG;
  if (k > 0 && (!values || !sums)) return MT_ERR_INVALID_ARG;
  if (n == 0) return MT_OK;
  bin_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(dirs, n, values, k, nside, nest, sums, counts,
                                                           (long long*)ipix);
  return cudaGetLastError() == cudaSuccess ? MT_OK : MT_ERR_CUDA;
}

extern "C" mt_status mt_deflection(const mt_octree* tree, const mt_trace_params* params, const double* dirs,
                                   int64_t n_rays, const double* xi, double* alpha, void* stream) {
  if (!tree) return MT_ERR_INVALID_ARG;
  mt_status st = check_trace_params(params, n_rays);
  if (st != MT_OK) return st;
  if (n_rays > 0 && (!dirs || !xi || !alpha)) return MT_ERR_INVALID_ARG;
  if (n_rays == 0) return MT_OK;
  DevCones C;
  fill_cones(tree, params, &C);
  deflection_kernel<<<grid_for(n_rays), 256, 0, (cudaStream_t)stream>>>(C, dirs, xi, n_rays, alpha);
  return cudaGetLastError() == cudaSuccess ? MT_OK : MT_ERR_CUDA;
}
