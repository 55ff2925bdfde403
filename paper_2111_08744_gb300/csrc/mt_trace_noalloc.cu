// mt_trace_rays_noalloc: the trace of mt_trace_rays with no device allocation at all.
//
// Its scratch -- the ray-queue counter and the cone table (observer, stop time and first
// ray of every cone) -- lives in one file-scope device array that is part of this
// library's image, so every GPU that loads the library holds it (about 160 KiB) until
// the process exits.  Host code cannot pass the array's name to a kernel: on the host
// that name is only a stand-in for the symbol, and a kernel given it would fault or, on
// systems where the GPU can reach host memory, quietly read and write the wrong memory.
// The device address is therefore fetched once per device with cudaGetSymbolAddress
// (with that device current) and passed to the kernel.
//
// Every call shares the one array: the queue counter is cleared and the cone table
// rewritten by each call on the caller's stream, so calls that overlap on the GPU race.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "mt_trace_device.cuh"

namespace mt {
namespace {

constexpr int kNoAllocMaxCones = MT_NOALLOC_MAX_CONES;
constexpr int kHeaderWords = 32;  // [0] ray-queue counter, rest reserved (keeps the table 256-B aligned)
constexpr int kBeginOff = kHeaderWords;                      // long long [max + 1]
constexpr int kObsOff = kBeginOff + kNoAllocMaxCones + 1;    // double [max][3]
constexpr int kStopOff = kObsOff + 3 * kNoAllocMaxCones;     // double [max]
constexpr int kScratchWords = kStopOff + kNoAllocMaxCones;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kScratchWords];

std::mutex g_mu;
unsigned long long* g_scratch_addr[kMaxDevices];  // device address of g_noalloc_scratch per device
unsigned long long g_host_table[kScratchWords - kHeaderWords];  // staging of the cone table (host)

template <class T, int IP>
__global__ void __launch_bounds__(kBlock, 4) trace_kernel_noalloc(DevField F, int n_cones, const double* __restrict__ dirs,
                                                               OutPtrs O, TraceArgs A, unsigned long long* scratch,
                                                               unsigned* err) {
  const long long* begin = (const long long*)(scratch + kBeginOff);
  const double* obs = (const double*)(scratch + kObsOff);
  const double* stop = (const double*)(scratch + kStopOff);
  const unsigned lane = threadIdx.x & 31u;
  const long long n = A.n_rays;
  const bool grav = A.gravity_on != 0;
  RayState r;
  long long ray = -1;
  bool exhausted = false;
  for (;;) {
    const bool need = (ray < 0) && !exhausted;
    const unsigned m = __ballot_sync(0xffffffffu, need);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned long long base = 0;
      if ((int)lane == leader) base = atomicAdd(scratch, (unsigned long long)__popc(m));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (need) {
        const long long id = (long long)base + __popc(m & ((1u << lane) - 1u));
        if (id < n) {
          ray = id;
          // cone c with begin[c] <= ray < begin[c + 1] (binary search; empty cones skipped)
          int lo = 0, hi = n_cones;
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (begin[mid] <= ray) lo = mid; else hi = mid;
          }
          r = ray_start<T>(F, obs + 3 * lo, stop[lo], dirs, n, ray, grav, err);
        } else {
          exhausted = true;
        }
      }
    }
    const bool alive = ray >= 0;
    if (!__any_sync(0xffffffffu, alive)) break;
    if (alive) {
      if (ray_step<T, IP>(F, A, r, err)) {
        ray_finish<T>(F, A, r, ray, n, O, err);
        ray = -1;
      }
    }
  }
}

template <class T, int IP>
int noalloc_blocks_per_sm() {
  static int cached = -1;
  if (cached < 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, trace_kernel_noalloc<T, IP>, kBlock, 0) != cudaSuccess ||
        b < 1)
      b = 1;
    cached = b;
  }
  return cached;
}

template <class T, int IP>
void launch_noalloc(const mt_octree* tree, int n_cones, const double* dirs, const OutPtrs& O, const TraceArgs& A,
                    unsigned long long* scratch, unsigned* err, cudaStream_t stream) {
  const int grid = tree->num_sms * noalloc_blocks_per_sm<T, IP>();
  trace_kernel_noalloc<T, IP><<<grid, kBlock, 0, stream>>>(launch_field(tree, A), n_cones, dirs, O, A, scratch, err);
}

template <class T>
void launch_noalloc_scheme(const mt_octree* tree, int n_cones, const double* dirs, const OutPtrs& O,
                           const TraceArgs& A, unsigned long long* scratch, unsigned* err, cudaStream_t stream) {
  switch (A.interp) {
    case MT_INTERP_NGP: launch_noalloc<T, MT_INTERP_NGP>(tree, n_cones, dirs, O, A, scratch, err, stream); break;
    case MT_INTERP_TSC: launch_noalloc<T, MT_INTERP_TSC>(tree, n_cones, dirs, O, A, scratch, err, stream); break;
    default: launch_noalloc<T, MT_INTERP_CIC>(tree, n_cones, dirs, O, A, scratch, err, stream); break;
  }
}

mt_status check_noalloc_params(const mt_trace_params* p, int64_t n_rays) {
  if (!p || n_rays < 0) return MT_ERR_INVALID_ARG;
  if (p->n_cones < 1 || p->steps_per_cell < 1 || p->max_steps < 1) return MT_ERR_INVALID_ARG;
  if (p->interp < MT_INTERP_CIC || p->interp > MT_INTERP_TSC) return MT_ERR_INVALID_ARG;
  if (p->n_cones > kNoAllocMaxCones) return MT_ERR_UNSUPPORTED;
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

}  // namespace
}  // namespace mt

using namespace mt;

extern "C" mt_status mt_trace_rays_noalloc(const mt_octree* tree, const mt_trace_params* params, const double* dirs,
                                           int64_t n_rays, const mt_ray_out* out, void* stream_) {
  if (!tree || !out) return MT_ERR_INVALID_ARG;
  mt_status st = check_noalloc_params(params, n_rays);
  if (st != MT_OK) return st;
  if (n_rays > 0 && !dirs) return MT_ERR_INVALID_ARG;
  if (n_rays == 0) return MT_OK;
  if (tree->device < 0 || tree->device >= kMaxDevices) return MT_ERR_UNSUPPORTED;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != tree->device && cudaSetDevice(tree->device) != cudaSuccess) return MT_ERR_CUDA;
  cudaStream_t stream = (cudaStream_t)stream_;
  cudaError_t e = cudaSuccess;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    // one-time set-up on this device (the octree's device is current here)
    if (!g_scratch_addr[tree->device]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e == cudaSuccess && p) g_scratch_addr[tree->device] = (unsigned long long*)p;
      else if (e == cudaSuccess) e = cudaErrorInvalidSymbol;
    }
    unsigned long long* scratch = g_scratch_addr[tree->device];
    if (e == cudaSuccess) {
      // cone table: first rays, observers, stop times
      const int nc = params->n_cones;
      long long* begin = (long long*)g_host_table;
      double* obs = (double*)(g_host_table + (kObsOff - kHeaderWords));
      double* stop = (double*)(g_host_table + (kStopOff - kHeaderWords));
      for (int c = 0; c <= nc; ++c) begin[c] = params->ray_begin[c];
      for (int c = 0; c < nc; ++c) {
        for (int d = 0; d < 3; ++d) obs[3 * c + d] = params->observer[3 * c + d];
        stop[c] = host_eta_stop(tree, params->z_max[c]);
      }
      // the queue counter must start at zero on every call
      e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long), stream);
      // a pageable-source copy returns once the staging table has been consumed
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(scratch + kBeginOff, begin, sizeof(long long) * (nc + 1), cudaMemcpyHostToDevice, stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(scratch + kObsOff, obs, sizeof(double) * 3 * nc, cudaMemcpyHostToDevice, stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(scratch + kStopOff, stop, sizeof(double) * nc, cudaMemcpyHostToDevice, stream);
    }
    if (e == cudaSuccess) {
      OutPtrs O = {out->x, out->k, out->eta, out->lambda, out->chi, out->path, out->z0, out->z1, out->z4, out->z5,
                   out->d_a, out->d_l, out->phi_o, out->phi_s, out->isw, out->n_steps, out->level, out->status, out->xi};
      TraceArgs A;
      A.steps_per_cell = params->steps_per_cell;
      A.interp = params->interp;
      A.ray_chunk = 32;
      A.gravity_on = params->gravity_on ? 1 : 0;
      A.max_steps = params->max_steps;
      A.n_rays = n_rays;
      unsigned* err = (unsigned*)(tree->ws + 1);  // the octree's status word, read by mt_device_status
      if (tree->precision == MT_FIELD_FP64) {
        launch_noalloc_scheme<double>(tree, params->n_cones, dirs, O, A, scratch, err, stream);
      } else {
        launch_noalloc_scheme<float>(tree, params->n_cones, dirs, O, A, scratch, err, stream);
      }
      e = cudaGetLastError();
    }
  }
  if (prev >= 0 && prev != tree->device) cudaSetDevice(prev);
  return e == cudaSuccess ? MT_OK : MT_ERR_CUDA;
}
