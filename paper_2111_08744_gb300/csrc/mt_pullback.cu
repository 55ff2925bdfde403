// build: fp64
// The field model of the differentiable form (documented at mt_pullback_coarse_phi in mt.h): its
// forward map (coarse potential -> records, mt_field_from_coarse_phi) and the pull-back of record
// cotangents to the coarse potential (its transpose, mt_pullback_coarse_phi).
//
//   records_0[c][s]  = w_s (phi_0[c], (D phi_0)[c])
//   records_l[c][s]  = w_s (I_0[phi_0](x_c), I_0[D phi_0](x_c)) + terms independent of phi_0
// with D the periodic 5-point central difference and I_0 trilinear interpolation of the
// periodic, cell-centred coarse grid at the refined cell's centre x_c.  Hence
//   dL/dphi_0 = A_phi + sum_d D_d^T A_d,   A = sum_s w_s (rbar_0 + sum_l I_0^T rbar_l),
// and D_d^T = -D_d for the antisymmetric periodic stencil.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "mt_internal.cuh"

namespace mt {
namespace {

__device__ __forceinline__ unsigned compact_bits3(unsigned long long v) {
  v &= 0x1249249249249249ull;
  v = (v | (v >> 2)) & 0x10c30c30c30c30c3ull;
  v = (v | (v >> 4)) & 0x100f00f00f00f00full;
  v = (v | (v >> 8)) & 0x1f0000ff0000ffull;
  v = (v | (v >> 16)) & 0x1f00000000ffffull;
  v = (v | (v >> 32)) & 0x1fffffull;
  return (unsigned)v;
}

struct SliceW {
  double w[kMaxSlices];
};

// A[c][q] = sum_s w_s rbar_0[c][s][q]
__global__ void coarse_accumulate(const double* __restrict__ r0, long long n0, int S, SliceW W, double* A) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n0; c += (long long)gridDim.x * blockDim.x)
    for (int q = 0; q < 4; ++q) {
      double a = 0.0;
      for (int s = 0; s < S; ++s) a += W.w[s] * r0[(c * S + s) * 4 + q];
      A[c * 4 + q] = a;
    }
}

// A += I_0^T (sum_s w_s rbar_l) for every cell of refined level l.
__global__ void refined_scatter(const double* __restrict__ rl, long long count, int S, SliceW W,
                                const unsigned long long* __restrict__ octkey, int l, int nc, double* A) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < count;
       r += (long long)gridDim.x * blockDim.x) {
    double a[4];
    bool any = false;
    for (int q = 0; q < 4; ++q) {
      double v = 0.0;
      for (int s = 0; s < S; ++s) v += W.w[s] * rl[(r * S + s) * 4 + q];
      a[q] = v;
      any = any || v != 0.0;
    }
    if (!any) continue;
    const unsigned long long key = (octkey[r >> 3] << 3) | (unsigned long long)(r & 7);
    const unsigned ci[3] = {compact_bits3(key), compact_bits3(key >> 1), compact_bits3(key >> 2)};
    long long i0[3];
    double f[3];
    const double inv = 1.0 / (double)(1 << l);
    for (int d = 0; d < 3; ++d) {
      const double u = ((double)ci[d] + 0.5) * inv - 0.5;  // coarse cell-centred coordinate
      const double fl = floor(u);
      i0[d] = (long long)fl;
      f[d] = u - fl;
    }
    for (int c = 0; c < 8; ++c) {
      const double w = ((c & 1) ? f[0] : 1.0 - f[0]) * ((c & 2) ? f[1] : 1.0 - f[1]) * ((c & 4) ? f[2] : 1.0 - f[2]);
      if (w == 0.0) continue;
      const unsigned x = (unsigned)((i0[0] + (c & 1)) & (nc - 1));
      const unsigned y = (unsigned)((i0[1] + ((c >> 1) & 1)) & (nc - 1));
      const unsigned z = (unsigned)((i0[2] + ((c >> 2) & 1)) & (nc - 1));
      double* dst = A + morton(x, y, z) * 4;
      for (int q = 0; q < 4; ++q)
        if (a[q] != 0.0) atomicAdd(dst + q, w * a[q]);
    }
  }
}

// dL/dphi_0[c] = A_phi[c] - sum_d (D_d A_d)[c]
__global__ void stencil_transpose(const double* __restrict__ A, long long n0, int nc, double inv12dx, double* out) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n0; c += (long long)gridDim.x * blockDim.x) {
    const unsigned long long key = (unsigned long long)c;
    const unsigned ci[3] = {compact_bits3(key), compact_bits3(key >> 1), compact_bits3(key >> 2)};
    double v = A[c * 4];
    for (int d = 0; d < 3; ++d) {
      double g[5];
      for (int o = -2; o <= 2; ++o) {
        unsigned p[3] = {ci[0], ci[1], ci[2]};
        p[d] = (unsigned)(((int)ci[d] + o) & (nc - 1));
        g[o + 2] = A[morton(p[0], p[1], p[2]) * 4 + 1 + d];
      }
      // D_d^T A_d = -(D_d A_d): -(A[-2] - 8 A[-1] + 8 A[+1] - A[+2]) / (12 dx)
      v -= (g[0] - 8.0 * g[1] + 8.0 * g[3] - g[4]) * inv12dx;
    }
    out[c] = v;
  }
}

// B[c] = (phi_0[c], (D phi_0)[c]) on the coarse grid (Morton order), D the periodic 5-point stencil.
__global__ void coarse_values(const double* __restrict__ phi0, long long n0, int nc, double inv12dx, double* B) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n0; c += (long long)gridDim.x * blockDim.x) {
    const unsigned long long key = (unsigned long long)c;
    const unsigned ci[3] = {compact_bits3(key), compact_bits3(key >> 1), compact_bits3(key >> 2)};
    B[c * 4] = phi0[c];
    for (int d = 0; d < 3; ++d) {
      double g[5];
      for (int o = -2; o <= 2; ++o) {
        unsigned p[3] = {ci[0], ci[1], ci[2]};
        p[d] = (unsigned)(((int)ci[d] + o) & (nc - 1));
        g[o + 2] = phi0[morton(p[0], p[1], p[2])];
      }
      B[c * 4 + 1 + d] = (g[0] - 8.0 * g[1] + 8.0 * g[3] - g[4]) * inv12dx;
    }
  }
}

// records_0[c][s] = w_s B[c] (+ base_0[c][s])
__global__ void coarse_records(const double* __restrict__ B, long long n0, int S, SliceW W,
                               const double* __restrict__ base, double* out) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n0; c += (long long)gridDim.x * blockDim.x)
    for (int s = 0; s < S; ++s)
      for (int q = 0; q < 4; ++q) {
        const long long i = (c * S + s) * 4 + q;
        out[i] = W.w[s] * B[c * 4 + q] + (base ? base[i] : 0.0);
      }
}

// records_l[r][s] = w_s I_0[B](x_r) (+ base_l[r][s]) for every cell r of refined level l, I_0 the
// trilinear interpolation of the periodic, cell-centred coarse grid at the cell's centre.
__global__ void refined_records(const double* __restrict__ B, long long count, int S, SliceW W,
                                const unsigned long long* __restrict__ octkey, int l, int nc,
                                const double* __restrict__ base, double* out) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < count;
       r += (long long)gridDim.x * blockDim.x) {
    const unsigned long long key = (octkey[r >> 3] << 3) | (unsigned long long)(r & 7);
    const unsigned ci[3] = {compact_bits3(key), compact_bits3(key >> 1), compact_bits3(key >> 2)};
    long long i0[3];
    double f[3];
    const double inv = 1.0 / (double)(1 << l);
    for (int d = 0; d < 3; ++d) {
      const double u = ((double)ci[d] + 0.5) * inv - 0.5;  // coarse cell-centred coordinate
      const double fl = floor(u);
      i0[d] = (long long)fl;
      f[d] = u - fl;
    }
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c = 0; c < 8; ++c) {
      const double w = ((c & 1) ? f[0] : 1.0 - f[0]) * ((c & 2) ? f[1] : 1.0 - f[1]) * ((c & 4) ? f[2] : 1.0 - f[2]);
      const unsigned x = (unsigned)((i0[0] + (c & 1)) & (nc - 1));
      const unsigned y = (unsigned)((i0[1] + ((c >> 1) & 1)) & (nc - 1));
      const unsigned z = (unsigned)((i0[2] + ((c >> 2) & 1)) & (nc - 1));
      const double* src = B + morton(x, y, z) * 4;
      for (int q = 0; q < 4; ++q) v[q] += w * src[q];
    }
    for (int s = 0; s < S; ++s)
      for (int q = 0; q < 4; ++q) {
        const long long i = (r * S + s) * 4 + q;
        out[i] = W.w[s] * v[q] + (base ? base[i] : 0.0);
      }
  }
}

}  // namespace
}  // namespace mt

using namespace mt;

extern "C" mt_status mt_field_from_coarse_phi(const mt_octree* tree, const double* phi0, const double* slice_weight,
                                              const double* const* base, double* const* records, void* stream_) {
  if (!tree || !phi0 || !slice_weight || !records) return MT_ERR_INVALID_ARG;
  for (int l = 0; l <= tree->n_levels; ++l)
    if (!records[l] && tree->count[l] > 0) return MT_ERR_INVALID_ARG;
  SliceW W;
  for (int s = 0; s < tree->n_slices; ++s) {
    if (!std::isfinite(slice_weight[s])) return MT_ERR_INVALID_ARG;
    W.w[s] = slice_weight[s];
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != tree->device && cudaSetDevice(tree->device) != cudaSuccess) return MT_ERR_CUDA;
  cudaStream_t stream = (cudaStream_t)stream_;
  const int nc = tree->f.nc;
  const long long n0 = (long long)nc * nc * nc;
  double* B = nullptr;
  cudaError_t e = cudaMalloc(&B, sizeof(double) * 4 * n0);
  if (e == cudaSuccess) {
    const int S = tree->n_slices;
    const int b0 = (int)std::min<long long>((n0 + 255) / 256, 65535ll * 8);
    coarse_values<<<b0, 256, 0, stream>>>(phi0, n0, nc, 1.0 / (12.0 * tree->f.dx0), B);
    coarse_records<<<b0, 256, 0, stream>>>(B, n0, S, W, base ? base[0] : nullptr, records[0]);
    for (int l = 1; l <= tree->n_levels; ++l) {
      const long long cnt = tree->count[l];
      if (cnt == 0) continue;
      const int b = (int)std::min<long long>((cnt + 255) / 256, 65535ll * 8);
      refined_records<<<b, 256, 0, stream>>>(B, cnt, S, W, tree->octkey[l], l, nc, base ? base[l] : nullptr,
                                             records[l]);
    }
    e = cudaGetLastError();
    cudaError_t e2 = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) e = e2;
    cudaFree(B);
  }
  if (prev >= 0 && prev != tree->device) cudaSetDevice(prev);
  if (e == cudaErrorMemoryAllocation) return MT_ERR_OOM;
  return e == cudaSuccess ? MT_OK : MT_ERR_CUDA;
}

extern "C" mt_status mt_pullback_coarse_phi(const mt_octree* tree, double* const* dL_drec, const double* slice_weight,
                                            double* dL_dphi0, void* stream_) {
  if (!tree || !dL_drec || !slice_weight || !dL_dphi0 || !dL_drec[0]) return MT_ERR_INVALID_ARG;
  SliceW W;
  for (int s = 0; s < tree->n_slices; ++s) {
    if (!std::isfinite(slice_weight[s])) return MT_ERR_INVALID_ARG;
    W.w[s] = slice_weight[s];
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != tree->device && cudaSetDevice(tree->device) != cudaSuccess) return MT_ERR_CUDA;
  cudaStream_t stream = (cudaStream_t)stream_;
  const int nc = tree->f.nc;
  const long long n0 = (long long)nc * nc * nc;
  double* A = nullptr;
  cudaError_t e = cudaMalloc(&A, sizeof(double) * 4 * n0);
  if (e == cudaSuccess) {
    const int S = tree->n_slices;
    const int b0 = (int)std::min<long long>((n0 + 255) / 256, 65535ll * 8);
    coarse_accumulate<<<b0, 256, 0, stream>>>(dL_drec[0], n0, S, W, A);
    for (int l = 1; l <= tree->n_levels; ++l) {
      const long long cnt = tree->count[l];
      if (cnt == 0 || !dL_drec[l]) continue;
      const int b = (int)std::min<long long>((cnt + 255) / 256, 65535ll * 8);
      refined_scatter<<<b, 256, 0, stream>>>(dL_drec[l], cnt, S, W, tree->octkey[l], l, nc, A);
    }
    stencil_transpose<<<b0, 256, 0, stream>>>(A, n0, nc, 1.0 / (12.0 * tree->f.dx0), dL_dphi0);
    e = cudaGetLastError();
    cudaError_t e2 = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) e = e2;
    cudaFree(A);
  }
  if (prev >= 0 && prev != tree->device) cudaSetDevice(prev);
  if (e == cudaErrorMemoryAllocation) return MT_ERR_OOM;
  return e == cudaSuccess ? MT_OK : MT_ERR_CUDA;
}
