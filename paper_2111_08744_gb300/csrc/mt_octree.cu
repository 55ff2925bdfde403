// Octree construction and lifetime (Sect. 2.1: flattened AMR, full-tree check).
//
// mt_build_octree copies (or borrows) the per-level records, validates the full-tree
// rule on the device (sorted keys, complete octets, parent present), and inserts every
// refined octet into its level's open-addressing hash, parent key -> octet index.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>

#include "mt_internal.cuh"

namespace mt {

namespace {

__global__ void check_dense_keys(const unsigned long long* keys, long long n, unsigned* bad) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (keys[i] != (unsigned long long)i) atomicOr(bad, kErrTree);
}

// One thread per key of refined level l: sortedness, octet completeness, key range,
// parent presence on level l-1, and hash insertion of each octet's parent key.
__global__ void build_level(const unsigned long long* keys, long long n, int key_bits, HashTable self,
                            ulonglong2* slots, HashTable parent_level, int parent_is_coarse, unsigned long long* octkey,
                            unsigned* bad) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long k = keys[i];
    const unsigned long long first = keys[i & ~7ll];
    bool ok = ((first & 7ull) == 0ull) && (k == (first | (unsigned long long)(i & 7)));
    if (i > 0) ok = ok && (keys[i - 1] < k);
    if (key_bits < 64) ok = ok && ((k >> key_bits) == 0ull);
    if (!ok) {
      atomicOr(bad, kErrTree);
      continue;
    }
    if ((i & 7) != 0) continue;
    const unsigned long long pk = k >> 3;  // parent key on level l-1
    octkey[i >> 3] = pk;
    if (!parent_is_coarse) {
      if (hash_find(parent_level, pk >> 3, bad) < 0) atomicOr(bad, kErrTree);
    }
    // insert pk -> octet index i / 8
    unsigned long long h = (pk * kHashMul) >> self.shift;
    bool done = false;
    for (unsigned long long probe = 0; probe <= self.mask && !done; ++probe) {
      unsigned long long prev = atomicCAS(&slots[h].x, kEmptyKey, pk);
      if (prev == kEmptyKey) {
        slots[h].y = (unsigned long long)(i >> 3);
        done = true;
      } else if (prev == pk) {
        atomicOr(bad, kErrTree);  // duplicate octet
        done = true;
      } else {
        h = (h + 1) & self.mask;
      }
    }
    if (!done) atomicOr(bad, kErrOOB);
  }
}

// Bitmap of coarse cells that have children (the parents of level-1 octets).
__global__ void mark_refined(const unsigned long long* octkey, long long n_oct, unsigned* bits) {
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n_oct; o += (long long)gridDim.x * blockDim.x) {
    const unsigned long long pk = octkey[o];
    atomicOr(&bits[pk >> 5], 1u << (pk & 31ull));
  }
}

int ilog2_exact(long long v) {
  int b = 0;
  while ((1ll << b) < v) ++b;
  return ((1ll << b) == v) ? b : -1;
}

void release(mt_octree* t) {
  if (!t) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(t->device);
  for (int l = 0; l <= kMaxLevels; ++l) {
    if (t->rec_alloc[l]) cudaFree(t->rec_alloc[l]);
    if (t->hash_alloc[l]) cudaFree(t->hash_alloc[l]);
    if (t->octkey[l]) cudaFree(t->octkey[l]);
  }
  if (t->bg_dev) cudaFree(t->bg_dev);
  if (t->refbits) cudaFree(t->refbits);
  if (t->bgf_dev) cudaFree(t->bgf_dev);
  if (t->ws) cudaFree(t->ws);
  std::free(t->bg_host);
  if (prev >= 0) cudaSetDevice(prev);
  delete t;
}

mt_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return MT_OK;
  return e == cudaErrorMemoryAllocation ? MT_ERR_OOM : MT_ERR_CUDA;
}

}  // namespace

void host_bg_eval(const double* tab, int n, double eta, double* a, double* H) {
  // node interval holding eta (eta_j <= eta < eta_{j+1}, clamped), as the device's bg_interval
  const double e0 = tab[0];
  const double de = (tab[4 * (n - 1)] - e0) / (double)(n - 1);
  double jf = std::floor((eta - e0) / de);
  jf = std::fmin(std::fmax(jf, 0.0), (double)(n - 2));
  int j = (int)jf;
  if (j > 0 && eta < tab[4 * j]) {
    --j;
  } else if (j < n - 2 && !(eta < tab[4 * (j + 1)])) {
    ++j;
  }
  const double* p = tab + 4 * j;
  const double* q = p + 4;
  const double d = q[0] - p[0];
  const double t = (eta - p[0]) / d;
  double t2 = t * t, t3 = t2 * t;
  double h00 = 2.0 * t3 - 3.0 * t2 + 1.0, h10 = t3 - 2.0 * t2 + t, h01 = -2.0 * t3 + 3.0 * t2, h11 = t3 - t2;
  if (a) *a = h00 * p[1] + h10 * d * (p[1] * p[2]) + h01 * q[1] + h11 * d * (q[1] * q[2]);
  if (H) *H = h00 * p[2] + h10 * d * p[3] + h01 * q[2] + h11 * d * q[3];
}

// eta at which a(eta) = 1/(1+z): bisection on the (monotone) background interpolant.
double host_eta_stop(const mt_octree* t, double z) {
  const double target = 1.0 / (1.0 + z);
  double lo = t->bg_host[0], hi = t->bg_host[4 * (t->bg_n - 1)];
  double ahi;
  host_bg_eval(t->bg_host, t->bg_n, hi, &ahi, nullptr);
  if (target >= ahi) return hi;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    double am;
    host_bg_eval(t->bg_host, t->bg_n, mid, &am, nullptr);
    if (am < target) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

}  // namespace mt

using namespace mt;

extern "C" mt_status mt_build_octree(const mt_grid_desc* grid, const mt_level_data* levels, const double* bg_table,
                                     int32_t bg_n, void* stream_, mt_octree** out) {
  if (!out) return MT_ERR_INVALID_ARG;
  *out = nullptr;
  if (!grid || !levels || !bg_table) return MT_ERR_INVALID_ARG;
  const int L = grid->n_levels, S = grid->n_slices, nc = grid->n_coarse;
  if (!(grid->box > 0.0) || !std::isfinite(grid->box)) return MT_ERR_INVALID_ARG;
  if (L < 0 || L > kMaxLevels || S < 1 || S > kMaxSlices) return MT_ERR_INVALID_ARG;
  const int bits0 = ilog2_exact(nc);
  if (nc < 1 || bits0 < 0 || bits0 > 20 || bits0 + L > 21) return MT_ERR_INVALID_ARG;
  if (grid->precision != MT_FIELD_FP64 && grid->precision != MT_FIELD_FP32) return MT_ERR_INVALID_ARG;
  if (!grid->slice_eta) return MT_ERR_INVALID_ARG;
  for (int s = 0; s < S; ++s) {
    if (!std::isfinite(grid->slice_eta[s])) return MT_ERR_INVALID_ARG;
    if (s > 0 && !(grid->slice_eta[s] > grid->slice_eta[s - 1])) return MT_ERR_INVALID_ARG;
  }
  if (bg_n < 2) return MT_ERR_INVALID_ARG;
  const double de = (bg_table[4 * (bg_n - 1)] - bg_table[0]) / (double)(bg_n - 1);
  if (!(de > 0.0)) return MT_ERR_INVALID_ARG;
  for (int j = 0; j < bg_n; ++j) {
    for (int q = 0; q < 4; ++q)
      if (!std::isfinite(bg_table[4 * j + q])) return MT_ERR_INVALID_ARG;
    if (std::fabs(bg_table[4 * j] - (bg_table[0] + de * j)) > 1e-9 * std::fabs(de) * bg_n) return MT_ERR_INVALID_ARG;
    if (!(bg_table[4 * j + 1] > 0.0)) return MT_ERR_INVALID_ARG;
  }
  const long long n0 = (long long)nc * nc * nc;
  if (levels[0].count != n0 || !levels[0].records) return MT_ERR_INVALID_ARG;
  for (int l = 0; l <= L; ++l)  // the kernels address a level's records by 32-bit row
    if (levels[l].count > (1ll << 32)) return MT_ERR_INVALID_ARG;
  for (int l = 1; l <= L; ++l) {
    if (levels[l].count < 0 || (levels[l].count & 7) != 0) return MT_ERR_NOT_FULL_TREE;
    if (levels[l].count > 0 && (!levels[l].keys || !levels[l].records)) return MT_ERR_INVALID_ARG;
  }
  for (int l = 0; l <= L; ++l)
    if (levels[l].residency < MT_HOST || levels[l].residency > MT_DEVICE_BORROW) return MT_ERR_INVALID_ARG;

  cudaStream_t stream = (cudaStream_t)stream_;
  mt_octree* t = new (std::nothrow) mt_octree;
  if (!t) return MT_ERR_OOM;
  std::memset(t, 0, sizeof(*t));
  if (cudaGetDevice(&t->device) != cudaSuccess) {
    delete t;
    return MT_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&t->num_sms, cudaDevAttrMultiProcessorCount, t->device);
  t->precision = grid->precision;
  t->n_levels = L;
  t->n_slices = S;
  const size_t rec_elem = (grid->precision == MT_FIELD_FP64 ? sizeof(double) : sizeof(float)) * 4;
  DevField& F = t->f;
  F.box = grid->box;
  F.nc = nc;
  F.L = L;
  F.S = S;
  F.periodic = grid->periodic ? 1 : 0;
  F.dx0 = grid->box / (double)nc;
  F.inv_dx0 = (double)nc / grid->box;
  for (int s = 0; s < S; ++s) F.seta[s] = grid->slice_eta[s];
  mt_status st = MT_OK;
  unsigned* d_bad = nullptr;
  unsigned long long* d_keys_tmp = nullptr;

#define MT_TRY(expr)                  \
  do {                                \
    cudaError_t e_ = (expr);          \
    if (e_ != cudaSuccess) {          \
      st = from_cuda(e_);             \
      goto fail;                      \
    }                                 \
  } while (0)

  MT_TRY(cudaMalloc(&t->ws, 64));
  MT_TRY(cudaMemsetAsync(t->ws, 0, 64, stream));
  MT_TRY(cudaMalloc(&d_bad, sizeof(unsigned)));
  MT_TRY(cudaMemsetAsync(d_bad, 0, sizeof(unsigned), stream));
  t->device_bytes = 64;

  // background table
  t->bg_n = bg_n;
  t->bg_host = (double*)std::malloc(sizeof(double) * 4 * bg_n);
  if (!t->bg_host) {
    st = MT_ERR_OOM;
    goto fail;
  }
  std::memcpy(t->bg_host, bg_table, sizeof(double) * 4 * bg_n);
  MT_TRY(cudaMalloc(&t->bg_dev, sizeof(double) * 4 * bg_n));
  MT_TRY(cudaMemcpyAsync(t->bg_dev, bg_table, sizeof(double) * 4 * bg_n, cudaMemcpyHostToDevice, stream));
  t->device_bytes += sizeof(double) * 4 * bg_n;
  F.bg = (const dvec4*)t->bg_dev;
  F.bg_n = bg_n;
  F.bg_eta0 = bg_table[0];
  F.bg_deta = de;
  F.bg_inv_deta = 1.0 / de;
  F.eta_o = bg_table[4 * (bg_n - 1)];
  {
    // single-precision Hermite table of H(eta) for the mixed path: node pairs (j, j+1)
    float* hf = (float*)std::malloc(sizeof(float) * 4 * bg_n);
    if (!hf) {
      st = MT_ERR_OOM;
      goto fail;
    }
    for (int j = 0; j < bg_n; ++j) {
      const int q = j + 1 < bg_n ? j + 1 : j;
      hf[4 * j + 0] = (float)bg_table[4 * j + 2];
      hf[4 * j + 1] = (float)(de * bg_table[4 * j + 3]);
      hf[4 * j + 2] = (float)bg_table[4 * q + 2];
      hf[4 * j + 3] = (float)(de * bg_table[4 * q + 3]);
    }
    cudaError_t e1 = cudaMalloc(&t->bgf_dev, sizeof(float4) * bg_n);
    if (e1 == cudaSuccess) e1 = cudaMemcpy(t->bgf_dev, hf, sizeof(float4) * bg_n, cudaMemcpyHostToDevice);
    std::free(hf);
    MT_TRY(e1);
    t->device_bytes += sizeof(float4) * bg_n;
  }
  F.bgf = t->bgf_dev;
  F.nf = nc << L;
  F.inv_dxf = (double)F.nf / grid->box;
  F.inv_dxf_f = (float)F.inv_dxf;
  F.dx0_f = (float)F.dx0;
  F.bg_inv_deta_f = (float)(1.0 / de);
  for (int s = 0; s + 1 < S; ++s) F.inv_dseta[s] = (float)(1.0 / (grid->slice_eta[s + 1] - grid->slice_eta[s]));
  for (int s = 0; s < S; ++s) F.seta_rel_f[s] = (float)(grid->slice_eta[s] - F.bg_eta0);

  for (int l = 0; l <= L; ++l) {
    const long long n = levels[l].count;
    t->count[l] = n;
    const size_t bytes = (size_t)n * S * rec_elem;
    if (n == 0) {
      // an empty refined level still gets a valid (empty) hash table, so every probe terminates
      MT_TRY(cudaMalloc(&t->hash_alloc[l], sizeof(ulonglong2) * 16));
      MT_TRY(cudaMemsetAsync(t->hash_alloc[l], 0xff, sizeof(ulonglong2) * 16, stream));
      F.hash[l].slots = t->hash_alloc[l];
      F.hash[l].mask = 15ull;
      F.hash[l].shift = 60;
      continue;
    }
    // records
    if (levels[l].residency == MT_DEVICE_BORROW) {
      F.rec[l] = levels[l].records;
    } else {
      MT_TRY(cudaMalloc(&t->rec_alloc[l], bytes));
      MT_TRY(cudaMemcpyAsync(t->rec_alloc[l], levels[l].records, bytes,
                             levels[l].residency == MT_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                             stream));
      F.rec[l] = t->rec_alloc[l];
      t->device_bytes += bytes;
    }
    // keys on the device for validation
    const unsigned long long* dkeys = nullptr;
    if (levels[l].keys) {
      if (levels[l].residency == MT_HOST) {
        if (d_keys_tmp) {
          MT_TRY(cudaStreamSynchronize(stream));
          cudaFree(d_keys_tmp);
          d_keys_tmp = nullptr;
        }
        MT_TRY(cudaMalloc(&d_keys_tmp, sizeof(unsigned long long) * n));
        MT_TRY(cudaMemcpyAsync(d_keys_tmp, levels[l].keys, sizeof(unsigned long long) * n, cudaMemcpyHostToDevice,
                               stream));
        dkeys = d_keys_tmp;
      } else {
        dkeys = (const unsigned long long*)levels[l].keys;
      }
    }
    const int blocks = (int)std::min<long long>((n + 255) / 256, 65535ll * 8);
    if (l == 0) {
      if (dkeys) check_dense_keys<<<blocks, 256, 0, stream>>>(dkeys, n, d_bad);
    } else {
      const long long n_oct = n / 8;
      long long cap = 16;
      while (cap < 2 * n_oct) cap <<= 1;
      int cap_bits = ilog2_exact(cap);
      MT_TRY(cudaMalloc(&t->hash_alloc[l], sizeof(ulonglong2) * cap));
      MT_TRY(cudaMemsetAsync(t->hash_alloc[l], 0xff, sizeof(ulonglong2) * cap, stream));
      t->device_bytes += sizeof(ulonglong2) * cap;
      F.hash[l].slots = t->hash_alloc[l];
      F.hash[l].mask = (unsigned long long)(cap - 1);
      F.hash[l].shift = 64 - cap_bits;
      const int key_bits = 3 * (bits0 + l);
      MT_TRY(cudaMalloc(&t->octkey[l], sizeof(unsigned long long) * n_oct));
      t->device_bytes += sizeof(unsigned long long) * n_oct;
      build_level<<<blocks, 256, 0, stream>>>(dkeys, n, key_bits, F.hash[l], t->hash_alloc[l], F.hash[l - 1],
                                              l == 1 ? 1 : 0, t->octkey[l], d_bad);
      if (l == 1) {
        const size_t words = (size_t)((n0 + 31) / 32);
        MT_TRY(cudaMalloc(&t->refbits, sizeof(unsigned) * words));
        MT_TRY(cudaMemsetAsync(t->refbits, 0, sizeof(unsigned) * words, stream));
        t->device_bytes += sizeof(unsigned) * words;
        mark_refined<<<(int)std::min<long long>((n_oct + 255) / 256, 65535ll * 8), 256, 0, stream>>>(
            t->octkey[1], n_oct, t->refbits);
        F.refbits = t->refbits;
      }
    }
    MT_TRY(cudaGetLastError());
  }
  {
    unsigned bad = 0;
    MT_TRY(cudaMemcpyAsync(&bad, d_bad, sizeof(unsigned), cudaMemcpyDeviceToHost, stream));
    MT_TRY(cudaStreamSynchronize(stream));
    if (bad & kErrTree) {
      st = MT_ERR_NOT_FULL_TREE;
      goto fail;
    }
    if (bad) {
      st = MT_ERR_OOB;
      goto fail;
    }
  }
  if (d_keys_tmp) cudaFree(d_keys_tmp);
  cudaFree(d_bad);
  *out = t;
  return MT_OK;
fail:
  cudaStreamSynchronize(stream);
  if (d_keys_tmp) cudaFree(d_keys_tmp);
  if (d_bad) cudaFree(d_bad);
  release(t);
  return st;
#undef MT_TRY
}

extern "C" void mt_free(mt_octree* tree) { release(tree); }

extern "C" mt_status mt_device_status(const mt_octree* tree, void* stream_) {
  if (!tree) return MT_ERR_INVALID_ARG;
  cudaStream_t stream = (cudaStream_t)stream_;
  unsigned long long flags = 0;
  if (cudaMemcpyAsync(&flags, tree->ws + 1, sizeof(flags), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
    return MT_ERR_CUDA;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return MT_ERR_CUDA;
  if (cudaMemsetAsync(tree->ws + 1, 0, sizeof(unsigned long long), stream) != cudaSuccess) return MT_ERR_CUDA;
  if (flags & kErrOOB) return MT_ERR_OOB;
  if (flags & kErrTimeout) return MT_ERR_TIMEOUT;
  return MT_OK;
}

extern "C" mt_status mt_octree_info(const mt_octree* tree, int64_t* cells_per_level, int64_t* device_bytes) {
  if (!tree) return MT_ERR_INVALID_ARG;
  if (cells_per_level)
    for (int l = 0; l <= tree->n_levels; ++l) cells_per_level[l] = tree->count[l];
  if (device_bytes) *device_bytes = tree->device_bytes;
  return MT_OK;
}

extern "C" const char* mt_status_str(mt_status s) {
  switch (s) {
    case MT_OK: return "ok";
    case MT_ERR_INVALID_ARG: return "invalid argument";
    case MT_ERR_OOM: return "out of device memory";
    case MT_ERR_CUDA: return "CUDA runtime error";
    case MT_ERR_NOT_FULL_TREE: return "not a full octree (unsorted keys, incomplete octet or missing parent)";
    case MT_ERR_TIMEOUT: return "device iteration bound reached";
    case MT_ERR_OOB: return "device index check failed";
    case MT_ERR_UNSUPPORTED: return "unsupported request";
  }
  return "unknown status";
}
