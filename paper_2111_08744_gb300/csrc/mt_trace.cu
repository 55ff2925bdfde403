// build: precision-split
// Null-geodesic integration (Sect. 2.2): one ray per thread, persistent warps.
//
// Each warp keeps 32 rays in flight.  A lane whose ray has finished takes the next id of
// the warp's current chunk of kRayChunk consecutive ray ids; an empty chunk is refilled from a
// device-wide counter (one atomic per chunk).  Rays of very different step counts (AMR
// levels, cones to different z_max) keep the lanes busy until the queue is empty, and a warp's
// rays stay neighbours in the input order (HEALPix NESTED: nearby on the sky), so their field
// gathers share cache lines.
//
// Per RK4 stage: coarse coordinates -> most refined level (hash probes) -> CIC with
// level fallback -> geodesic right-hand side, Eqs. (2)-(4) (mt_trace_device.cuh).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "mt_trace_device.cuh"

namespace mt {

// Ray ids a warp claims at a time (TraceArgs::ray_chunk, a multiple of 32; default 32, one lane's
// worth per lane).  Larger chunks keep more of a warp's rays sky neighbours but leave warps holding
// unstarted rays at the end of the queue (a tail with the rest of the GPU idle).

template <class T>
__device__ void ray_init(const DevField& F, const DevCones& C, const double* __restrict__ dirs, long long n,
                         long long ray, bool grav, RayState& r, unsigned* err) {
  int c = 0;
  while (c + 1 < C.n && C.begin[c + 1] <= ray) ++c;
  r = ray_start<T>(F, C.obs[c], C.eta_stop[c], dirs, n, ray, grav, err);
}

// BS threads per block; the register budget (128 per thread) is the same for every block size.
// IP: the interpolation scheme (MT_INTERP_*), fixed per instantiation.  Staged (FP32 fields): each
// ray's CIC neighbourhood (TSC: its 27 neighbour rows) is staged in shared memory; otherwise the
// records are read through L1 at every stage.
template <class T, int BS, int IP, bool Staged = true>
__global__ void __launch_bounds__(BS, 512 / BS) trace_kernel(DevField F, DevCones C, const double* __restrict__ dirs,
                                                              OutPtrs O, TraceArgs A, unsigned long long* ws) {
  unsigned* err = (unsigned*)(ws + 1);
  const unsigned lane = threadIdx.x & 31u;
  const long long n = A.n_rays;
  const bool grav = A.gravity_on != 0;
  // mixed path: per-ray CIC neighbourhood staged in shared memory (16 float4 + keys per thread)
  extern __shared__ float4 smem[];
  LaneCache lc;
  lc.rec = smem + threadIdx.x;
  lc.key = (int4*)(smem + 16 * BS) + threadIdx.x;
  lc.stride = BS;
  lc.loc = (int4*)(smem + 16 * BS) + BS + threadIdx.x;
  lc.neg = (int4*)(smem + 16 * BS) + 2 * BS + threadIdx.x;
  if (sizeof(T) == 4 && Staged) {
    *lc.loc = make_int4(0, 0, 0, -1);
    lc.neg[0] = lc.neg[BS] = make_int4(-1, 0, 0, 0);
  }
  const LaneCache* lcp = (sizeof(T) == 4 && Staged) ? &lc : nullptr;
  const unsigned long long chunk = (unsigned long long)A.ray_chunk;
  RayState r;
  long long ray = -1;
  bool exhausted = false;
  unsigned long long pool = 0;  // next id of this warp's current chunk (warp-uniform)
  int pool_left = 0;            // ids left in it
  for (;;) {
    const bool need = (ray < 0) && !exhausted;
    const unsigned m = __ballot_sync(0xffffffffu, need);
    if (m) {
      const int leader = __ffs(m) - 1;
      const int k = __popc(m);
      const int from_pool = k < pool_left ? k : pool_left;
      unsigned long long fresh = 0;
      if (k > from_pool) {
        if ((int)lane == leader) fresh = atomicAdd(ws, chunk);
        fresh = __shfl_sync(0xffffffffu, fresh, leader);
      }
      const int rank = __popc(m & ((1u << lane) - 1u));
      const unsigned long long pick = rank < from_pool ? pool + rank : fresh + (rank - from_pool);
      if (k > from_pool) {
        pool = fresh + (k - from_pool);
        pool_left = (int)chunk - (k - from_pool);
      } else {
        pool += k;
        pool_left -= k;
      }
      if (need) {
        const long long id = (long long)pick;
        if (id < n) {
          ray = id;
          ray_init<T>(F, C, dirs, n, ray, grav, r, err);
          if (lcp) *lc.key = make_int4(-1, 0, 0, 0);
        } else {
          exhausted = true;
        }
      }
    }
    const bool alive = ray >= 0;
    if (!__any_sync(0xffffffffu, alive)) break;
    if (alive) {
      if (ray_step<T, IP>(F, A, r, err, lcp)) {
        ray_finish<T>(F, A, r, ray, n, O, err);
        ray = -1;
      }
    }
  }
}

// Dynamic shared memory of trace_kernel<T, BS, IP, Staged>: the mixed path's per-thread neighbourhood
// cache, last locate answer and two incomplete-neighbourhood keys (320 B per thread).
template <class T, int BS, bool Staged>
constexpr size_t trace_smem() {
  return (sizeof(T) == 4 && Staged) ? (size_t)BS * (16 * sizeof(float4) + 4 * sizeof(int4)) : 0;
}

template <class T, int BS, int IP, bool Staged>
int blocks_per_sm() {
  static int cached = -1;
  if (cached < 0) {
    const size_t sm = trace_smem<T, BS, Staged>();
    if (sm > 48 * 1024)
      cudaFuncSetAttribute(trace_kernel<T, BS, IP, Staged>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, trace_kernel<T, BS, IP, Staged>, BS, sm) != cudaSuccess ||
        b < 1)
      b = 1;
    cached = b;
  }
  return cached;
}

template <class T, int BS, int IP, bool Staged = true>
void launch_trace_bs(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O,
                     const TraceArgs& A, cudaStream_t stream) {
  int bps = blocks_per_sm<T, BS, IP, Staged>();
  if (tree->launch_bps > 0 && tree->launch_bps < bps) bps = tree->launch_bps;
  trace_kernel<T, BS, IP, Staged><<<tree->num_sms * bps, BS, trace_smem<T, BS, Staged>(), stream>>>(
      launch_field(tree, A), C, dirs, O, A, tree->ws);
}

template <class T, bool Staged>
void launch_trace_cic(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O,
                      const TraceArgs& A, cudaStream_t stream) {
  switch (tree->launch_block) {
    case 64: launch_trace_bs<T, 64, MT_INTERP_CIC, Staged>(tree, C, dirs, O, A, stream); break;
    case 256: launch_trace_bs<T, 256, MT_INTERP_CIC, Staged>(tree, C, dirs, O, A, stream); break;
    default: launch_trace_bs<T, 128, MT_INTERP_CIC, Staged>(tree, C, dirs, O, A, stream); break;
  }
}

// Launch shape: the octree's configuration (mt_set_launch_config, mt_set_trace_options), default 128
// threads, as many blocks per SM as fit, the staged neighbourhood.  NGP and TSC run with 128 threads
// per block, staged.
template <class T>
void launch_trace(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O, const TraceArgs& A,
                  cudaStream_t stream) {
  if (A.interp == MT_INTERP_NGP) {
    launch_trace_bs<T, 128, MT_INTERP_NGP>(tree, C, dirs, O, A, stream);
    return;
  }
  if (A.interp == MT_INTERP_TSC) {
    launch_trace_bs<T, 128, MT_INTERP_TSC>(tree, C, dirs, O, A, stream);
    return;
  }
  if constexpr (sizeof(T) == 4) {
    if (tree->staging == 2) {
      launch_trace_cic<T, false>(tree, C, dirs, O, A, stream);
      return;
    }
  }
  launch_trace_cic<T, true>(tree, C, dirs, O, A, stream);
}

#ifdef MT_TU_FP64
// FP64-field instantiations (this translation unit is compiled without FMA contraction).
void launch_trace_fp64(const mt_octree* tree, const DevCones& C, const double* dirs, const OutPtrs& O,
                       const TraceArgs& A, cudaStream_t stream) {
  launch_trace<double>(tree, C, dirs, O, A, stream);
}
#endif

}  // namespace mt

#ifndef MT_TU_FP64
using namespace mt;

namespace mt {

mt_status check_trace_params(const mt_trace_params* p, int64_t n_rays) {
  if (!p || n_rays < 0) return MT_ERR_INVALID_ARG;
  if (p->n_cones < 1 || p->n_cones > kMaxCones || p->steps_per_cell < 1 || p->max_steps < 1) return MT_ERR_INVALID_ARG;
  if (p->interp < MT_INTERP_CIC || p->interp > MT_INTERP_TSC) return MT_ERR_INVALID_ARG;
  if (!p->observer || !p->z_max || !p->ray_begin) return MT_ERR_INVALID_ARG;
  if (p->ray_begin[0] != 0 || p->ray_begin[p->n_cones] != n_rays) return MT_ERR_INVALID_ARG;
  for (int c = 0; c < p->n_cones; ++c) {
    if (p->ray_begin[c + 1] < p->ray_begin[c]) return MT_ERR_INVALID_ARG;
    if (!(p->z_max[c] >= 0.0) || !std::isfinite(p->z_max[c])) return MT_ERR_INVALID_ARG;
    for (int d = 0; d < 3; ++d)
      if (!std::isfinite(p->observer[3 * c + d])) return MT_ERR_INVALID_ARG;
  }
  return MT_OK;
}

void fill_cones(const mt_octree* tree, const mt_trace_params* params, DevCones* C) {
  C->n = params->n_cones;
  C->pad = 0;
  for (int c = 0; c < C->n; ++c) {
    C->begin[c] = params->ray_begin[c];
    for (int d = 0; d < 3; ++d) C->obs[c][d] = params->observer[3 * c + d];
    C->eta_stop[c] = host_eta_stop(tree, params->z_max[c]);
  }
  C->begin[C->n] = params->ray_begin[C->n];
}

}  // namespace mt

extern "C" mt_status mt_trace_rays(const mt_octree* tree, const mt_trace_params* params, const double* dirs,
                                   int64_t n_rays, const mt_ray_out* out, void* stream_) {
  if (!tree || !out) return MT_ERR_INVALID_ARG;
  mt_status st = check_trace_params(params, n_rays);
  if (st != MT_OK) return st;
  if (n_rays > 0 && !dirs) return MT_ERR_INVALID_ARG;
  if (n_rays == 0) return MT_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != tree->device && cudaSetDevice(tree->device) != cudaSuccess) return MT_ERR_CUDA;
  cudaStream_t stream = (cudaStream_t)stream_;
  DevCones C;
  fill_cones(tree, params, &C);
  OutPtrs O = {out->x, out->k, out->eta, out->lambda, out->chi, out->path, out->z0, out->z1, out->z4, out->z5,
               out->d_a, out->d_l, out->phi_o, out->phi_s, out->isw, out->n_steps, out->level, out->status, out->xi};
  TraceArgs A;
  A.steps_per_cell = params->steps_per_cell;
  A.interp = params->interp;
  A.ray_chunk = tree->ray_chunk > 0 ? tree->ray_chunk : 32;
  A.gravity_on = params->gravity_on ? 1 : 0;
  A.max_steps = params->max_steps;
  A.n_rays = n_rays;
  cudaError_t e = cudaMemsetAsync(tree->ws, 0, sizeof(unsigned long long), stream);
  if (e == cudaSuccess) {
    if (tree->precision == MT_FIELD_FP64) {
      launch_trace_fp64(tree, C, dirs, O, A, stream);
    } else {
      launch_trace<float>(tree, C, dirs, O, A, stream);
    }
    e = cudaGetLastError();
  }
  if (prev >= 0 && prev != tree->device) cudaSetDevice(prev);
  return e == cudaSuccess ? MT_OK : MT_ERR_CUDA;
}

extern "C" mt_status mt_set_launch_config(mt_octree* tree, int32_t block_size, int32_t blocks_per_sm) {
  if (!tree) return MT_ERR_INVALID_ARG;
  if (block_size != 0 && block_size != 64 && block_size != 128 && block_size != 256) return MT_ERR_INVALID_ARG;
  if (blocks_per_sm < 0) return MT_ERR_INVALID_ARG;
  tree->launch_block = block_size;
  tree->launch_bps = blocks_per_sm;
  return MT_OK;
}
extern "C" mt_status mt_set_trace_options(mt_octree* tree, int32_t ray_chunk, int32_t staging) {
  if (!tree) return MT_ERR_INVALID_ARG;
  if (ray_chunk != 0 && (ray_chunk < 32 || ray_chunk > 1024 || ray_chunk % 32 != 0)) return MT_ERR_INVALID_ARG;
  if (staging < 0 || staging > 2) return MT_ERR_INVALID_ARG;
  tree->ray_chunk = ray_chunk;
  tree->staging = staging;
  return MT_OK;
}
#endif  // MT_TU_FP64
