// Batched kernels for many independent 2D Euler problems of degree 3 or 4.
//
// Work is a list of tiles (problem, block): element tiles for the local and
// update phases, face-node tiles for the face phase.  Each tile copies its
// problem's parameters (mesh, buffers) into shared memory and runs the same
// block body as the single-problem kernels; the reference tables, which depend
// only on the degree, stay kernel parameters as in the single-problem kernels.
//
//   k_batch_local / k_batch_face / k_batch_update : one launch per phase over
//       the tiles of every problem (three launches per step for the batch).
//   k_batch_fused : one cooperative, persistent launch for all phases of
//       nsteps steps; blocks stride over the tiles and meet at a grid barrier
//       between phases.  The barrier's wait is bounded: after A.spin_limit
//       polls it sets the error flag and every block returns.
#include <cstdint>

#include "cr_batch.cuh"
#include "cr_launch.cuh"

namespace crk {
namespace {

using Eq2 = EqEuler<2>;

template <typename real>
struct SharedParams {
  static_assert(sizeof(KParams<real>) % 8 == 0, "parameter block copied as 8-byte words");
  static constexpr int kWords = int(sizeof(KParams<real>) / 8);
};

// Copy problem prob's parameters into shared memory (all threads; barriers
// around the copy because the previous tile's body may still read it).
template <typename real>
__device__ __forceinline__ void load_params(KParams<real>* sP, const KParams<real>* src) {
  __syncthreads();
  const unsigned long long* a = reinterpret_cast<const unsigned long long*>(src);
  unsigned long long* b = reinterpret_cast<unsigned long long*>(sP);
  for (int i = threadIdx.x; i < SharedParams<real>::kWords; i += blockDim.x) b[i] = a[i];
  __syncthreads();
}

template <typename real, int PHASE>
__device__ __forceinline__ void el_tile(const BatchArgs<real>& A, KParams<real>* sP, int t, int& cur) {
  constexpr bool MIXED = sizeof(real) == 4;
  const BatchTile tile = A.t_el[t];
  if (tile.prob != cur) {
    load_params(sP, A.P + tile.prob);
    cur = tile.prob;
  }
  if (A.deg[tile.prob] == 3) {
    if (PHASE == 0) local_body<2, 3, Eq2, real, MIXED>(*sP, A.tb[0], tile.blk);
    else update_body<2, 3, Eq2, real, MIXED>(*sP, A.tb[0], A.td[0], tile.blk, A.nblk_el[tile.prob]);
  } else {
    if (PHASE == 0) local_body<2, 4, Eq2, real, MIXED>(*sP, A.tb[1], tile.blk);
    else update_body<2, 4, Eq2, real, MIXED>(*sP, A.tb[1], A.td[1], tile.blk, A.nblk_el[tile.prob]);
  }
  __syncthreads();  // the next tile reuses the dynamic shared memory
}

template <typename real>
__device__ __forceinline__ void face_tile(const BatchArgs<real>& A, KParams<real>* sP, int t, int& cur) {
  const BatchTile tile = A.t_face[t];
  if (tile.prob != cur) {
    load_params(sP, A.P + tile.prob);
    cur = tile.prob;
  }
  if (A.deg[tile.prob] == 3) face_body<2, 3, Eq2, real>(*sP, tile.blk);
  else face_body<2, 4, Eq2, real>(*sP, tile.blk);
}

// Grid-wide barrier of a cooperative launch (all blocks resident).  Thread 0
// of each block arrives on bar[0]; the last of gridDim.x + phantom arrivals
// resets it and advances the generation bar[1]; the others poll the
// generation, at most spin_limit times.
__device__ bool grid_barrier(unsigned* bar, int* err, unsigned long long spin_limit, int phantom) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x + unsigned(phantom) - 1u) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned long long spins = 0;
      while (*gen == g) {
        if (++spins > spin_limit) {
          atomicOr(err, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *reinterpret_cast<volatile int*>(err) == 0;
}

// Resident blocks per SM: as the single-problem kernels (MinBlocks), scaled
// from 256-thread blocks to T threads.
template <typename real, int T, int PHASE>
struct BatchMinBlocks {
  static constexpr bool MIXED = sizeof(real) == 4;
  static constexpr int per256 = PHASE == 0 ? MinBlocks<MIXED>::local : MinBlocks<MIXED>::update;
  static constexpr int value = per256 * 256 / T;
};

template <typename real, int T>
__global__ void __launch_bounds__(T, (BatchMinBlocks<real, T, 0>::value)) k_batch_local(const __grid_constant__ BatchArgs<real> A) {
  __shared__ __align__(16) KParams<real> sP;
  int cur = -1;
  el_tile<real, 0>(A, &sP, blockIdx.x, cur);
}

template <typename real, int T>
__global__ void __launch_bounds__(T, (BatchMinBlocks<real, T, 2>::value)) k_batch_update(const __grid_constant__ BatchArgs<real> A) {
  __shared__ __align__(16) KParams<real> sP;
  int cur = -1;
  el_tile<real, 2>(A, &sP, blockIdx.x, cur);
}

template <typename real, int T>
__global__ void __launch_bounds__(T) k_batch_face(const __grid_constant__ BatchArgs<real> A) {
  __shared__ __align__(16) KParams<real> sP;
  int cur = -1;
  face_tile<real>(A, &sP, blockIdx.x, cur);
}

// Register budget of the persistent kernel: that of the largest body it runs,
// as in the single-problem kernels: 128 per thread in FP64 (two 256-thread
// blocks per SM), 64 in FP32 bulk (four; those bodies are latency bound and
// need the resident warps).
template <typename real, int T>
struct FusedMinBlocks {
  static constexpr int value = 65536 / (T * (sizeof(real) == 4 ? 64 : 128));
};

template <typename real, int T>
__global__ void __launch_bounds__(T, (FusedMinBlocks<real, T>::value)) k_batch_fused(const __grid_constant__ BatchArgs<real> A) {
  __shared__ __align__(16) KParams<real> sP;
  int cur = -1;
  // tiles by grid stride: blocks see every problem size and degree, which
  // balances the load better than contiguous runs of tiles (measured: 67.7
  // against 73.6 ms per step on the 96-problem ensemble)
  for (int s = 0; s < A.nsteps; ++s) {
    for (int t = blockIdx.x; t < A.n_el; t += gridDim.x) el_tile<real, 0>(A, &sP, t, cur);
    if (!grid_barrier(A.bar, A.err, A.spin_limit, A.phantom)) return;
    for (int t = blockIdx.x; t < A.n_face; t += gridDim.x) face_tile<real>(A, &sP, t, cur);
    if (!grid_barrier(A.bar, A.err, A.spin_limit, A.phantom)) return;
    for (int t = blockIdx.x; t < A.n_el; t += gridDim.x) el_tile<real, 2>(A, &sP, t, cur);
    if (!grid_barrier(A.bar, A.err, A.spin_limit, A.phantom)) return;
  }
}

template <typename real>
size_t smem_for(int threads) {
  constexpr bool MIXED = sizeof(real) == 4;
  using I3 = Impl<2, 3, Eq2, real, MIXED>;
  using I4 = Impl<2, 4, Eq2, real, MIXED>;
  const int s3 = (threads + I3::NP - 1) / I3::NP, s4 = (threads + I4::NP - 1) / I4::NP;
  size_t m = I3::smem_local(s3);
  m = m > I3::smem_update(s3) ? m : I3::smem_update(s3);
  m = m > I4::smem_local(s4) ? m : I4::smem_local(s4);
  m = m > I4::smem_update(s4) ? m : I4::smem_update(s4);
  return m;
}

template <typename real, int T>
cudaError_t configure_t() {
  const int sm = (int)smem_for<real>(T);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_batch_local<real, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
    return e;
  if ((e = cudaFuncSetAttribute(k_batch_update<real, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
    return e;
  return cudaFuncSetAttribute(k_batch_fused<real, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

template <typename real, int T>
cudaError_t launch_phase_t(int phase, const BatchArgs<real>& A, cudaStream_t s) {
  const size_t sm = smem_for<real>(T);
  if (phase == 0) {
    if (A.n_el > 0) k_batch_local<real, T><<<A.n_el, T, sm, s>>>(A);
  } else if (phase == 1) {
    if (A.n_face > 0) k_batch_face<real, T><<<A.n_face, T, 0, s>>>(A);
  } else {
    if (A.n_el > 0) k_batch_update<real, T><<<A.n_el, T, sm, s>>>(A);
  }
  return cudaGetLastError();
}

template <typename real, int T>
cudaError_t launch_fused_t(int grid, const BatchArgs<real>& A, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(T);
  cfg.dynamicSmemBytes = smem_for<real>(T);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_batch_fused<real, T>, A);
}

template <typename real, int T>
cudaError_t max_blocks_t(int* blocks) {
  int dev = 0, sms = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_fused<real, T>, T, smem_for<real>(T));
  *blocks = per * sms;
  return e;
}

template <typename real>
__global__ void k_batch_set_run(const KParams<real>* P, int n, double t_final) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  TimeCtl* c = P[i].b.ctl;
  c->t_final = t_final;
  c->dt_fixed = 0.0;
  plan_step(c);
}

}  // namespace

cudaError_t batch_set_run(const void* P, int n, double t_final, bool fp32, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (fp32)
    k_batch_set_run<float><<<(n + 127) / 128, 128, 0, s>>>(static_cast<const KParams<float>*>(P), n, t_final);
  else
    k_batch_set_run<double><<<(n + 127) / 128, 128, 0, s>>>(static_cast<const KParams<double>*>(P), n, t_final);
  return cudaGetLastError();
}

size_t batch_smem(int threads, bool fp32) {
  return fp32 ? smem_for<float>(threads) : smem_for<double>(threads);
}

cudaError_t batch_configure(int threads, bool fp32) {
  if (threads == 128) return fp32 ? configure_t<float, 128>() : configure_t<double, 128>();
  if (threads == 256) return fp32 ? configure_t<float, 256>() : configure_t<double, 256>();
  return cudaErrorInvalidValue;
}

cudaError_t batch_fused_max_blocks(int threads, bool fp32, int* blocks) {
  if (threads == 128) return fp32 ? max_blocks_t<float, 128>(blocks) : max_blocks_t<double, 128>(blocks);
  if (threads == 256) return fp32 ? max_blocks_t<float, 256>(blocks) : max_blocks_t<double, 256>(blocks);
  return cudaErrorInvalidValue;
}

cudaError_t batch_launch_phase(int threads, int phase, const void* args, bool fp32, cudaStream_t s) {
  if (fp32) {
    const BatchArgs<float>& A = *static_cast<const BatchArgs<float>*>(args);
    if (threads == 128) return launch_phase_t<float, 128>(phase, A, s);
    if (threads == 256) return launch_phase_t<float, 256>(phase, A, s);
  } else {
    const BatchArgs<double>& A = *static_cast<const BatchArgs<double>*>(args);
    if (threads == 128) return launch_phase_t<double, 128>(phase, A, s);
    if (threads == 256) return launch_phase_t<double, 256>(phase, A, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t batch_launch_fused(int threads, int grid, const void* args, bool fp32, cudaStream_t s) {
  if (fp32) {
    const BatchArgs<float>& A = *static_cast<const BatchArgs<float>*>(args);
    if (threads == 128) return launch_fused_t<float, 128>(grid, A, s);
    if (threads == 256) return launch_fused_t<float, 256>(grid, A, s);
  } else {
    const BatchArgs<double>& A = *static_cast<const BatchArgs<double>*>(args);
    if (threads == 128) return launch_fused_t<double, 128>(grid, A, s);
    if (threads == 256) return launch_fused_t<double, 256>(grid, A, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace crk
