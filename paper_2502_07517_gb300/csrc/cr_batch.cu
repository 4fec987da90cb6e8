// Batched kernels for many independent 2D Euler problems of degree 3 or 4.
//
// Work is a list of tiles (problem, block): element tiles for the local and
// update phases, face-node tiles for the face phase.  Each tile copies its
// problem's parameters (mesh, buffers) into shared memory and runs the same
// block body as the single-problem kernels; the reference tables, which depend
// only on the degree, stay kernel parameters as in the single-problem kernels.
//
//   k_batch_local_n / k_batch_face / k_batch_update_n (+ k_batch_finish, one warp
//       per problem ending its step) : one launch per phase
//       over the tiles of every problem (per degree for the element phases:
//       up to six launches per step for the batch).
//   k_batch_fused : one cooperative, persistent launch for all phases of
//       nsteps steps.  The work items (step, phase, tile) form one queue in
//       that order; blocks claim kFusedClaim * A.tiles consecutive items at a
//       time from an atomic counter (the next claim is made while the current
//       one runs).  There is no grid barrier: an item waits only for the work
//       of its own problem it reads (the previous phase of the same step, or
//       the previous step's update), counted per (phase, problem); a block
//       publishes its finished tiles before it waits.  Every item an item
//       waits for lies earlier in the queue and has been claimed by a running
//       block, so the waits always end; they are bounded all the same: after
//       A.spin_limit polls the block sets the error flag and returns, and
//       blocks that see the flag stop.
#include <cstddef>
#include <cstdint>

#include "cr_batch.cuh"
#include "cr_launch.cuh"

namespace crk {
namespace {

using Eq2 = EqEuler<2>;

// The part of a problem's parameter block the bodies read from shared memory:
// everything before the reference tables (the kernels take those per degree).
template <typename real>
struct SharedParams {
  static constexpr size_t kBytes = offsetof(KParams<real>, tb);
  static_assert(kBytes % 8 == 0, "parameter block copied as 8-byte words");
  static constexpr int kWords = int(kBytes / 8);
};

// Copy problem prob's parameters (all but the tables) into shared memory (all
// threads; barriers around the copy because the previous tile's body may still
// read it).
template <typename real>
__device__ __forceinline__ void load_params(KParams<real>* sP, const KParams<real>* src) {
  __syncthreads();
  const unsigned long long* a = reinterpret_cast<const unsigned long long*>(src);
  unsigned long long* b = reinterpret_cast<unsigned long long*>(sP);
  for (int i = threadIdx.x; i < SharedParams<real>::kWords; i += blockDim.x) b[i] = a[i];
  __syncthreads();
}

template <typename real, int PHASE, int T>
__device__ __forceinline__ void el_tile(const BatchArgs<real>& A, KParams<real>* sP, int t, int& cur) {
  constexpr bool MIXED = sizeof(real) == 4;
  const BatchTile tile = PHASE == 2 ? A.t_upd[t] : A.t_el[t];
  if (tile.prob != cur) {
    load_params(sP, A.P + tile.prob);
    cur = tile.prob;
  }
  if (A.deg[tile.prob] == 3) {
    if (PHASE == 0) local_body<2, 3, Eq2, real, MIXED, T>(*sP, A.tb[0], tile.blk);
    else update_body<2, 3, Eq2, real, MIXED, T>(*sP, A.tb[0], A.td[0], tile.blk, A.nblk_upd[tile.prob]);
  } else {
    if (PHASE == 0) local_body<2, 4, Eq2, real, MIXED, T>(*sP, A.tb[1], tile.blk);
    else update_body<2, 4, Eq2, real, MIXED, T>(*sP, A.tb[1], A.td[1], tile.blk, A.nblk_upd[tile.prob]);
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

// Resident blocks per SM: as the single-problem kernels (MinBlocks), scaled
// from 256-thread blocks to T threads.
template <typename real, int T, int PHASE>
struct BatchMinBlocks {
  static constexpr bool MIXED = sizeof(real) == 4;
  static constexpr int per256 = PHASE == 0 ? MinBlocks<MIXED>::local : MinBlocks<MIXED>::update;
  static constexpr int value = per256 * 256 / T;
};

// Phase kernels for the tiles of one degree N: blocks of exactly the whole
// elements that fit in T threads (TB threads, as the single-problem kernels),
// the body of that degree only.  One tile per block: a loop over several
// consecutive tiles per block was measured 15-25% slower on the 96-problem
// ensemble (48 against 55-61 ms per step), so the tiles per block apply to the
// fused kernel's claims only.
template <int N, int T> struct DegShape {
  static constexpr int NP = (N + 1) * (N + 1);
  static constexpr int EPB = T / NP;
  static constexpr int TB = EPB * NP;
};

template <typename real, int N, int T>
__global__ void __launch_bounds__(DegShape<N, T>::TB, (BatchMinBlocks<real, T, 0>::value)) k_batch_local_n(const __grid_constant__ BatchArgs<real> A) {
  __shared__ __align__(16) KParams<real> sP;
  constexpr bool MIXED = sizeof(real) == 4;
  const BatchTile tile = A.t_el[A.el_first[N - 3] + blockIdx.x];
  load_params(&sP, A.P + tile.prob);
  local_body<2, N, Eq2, real, MIXED, DegShape<N, T>::TB>(sP, A.tb[N - 3], tile.blk);
}

template <typename real, int N, int T>
__global__ void __launch_bounds__(DegShape<N, T>::TB, (BatchMinBlocks<real, T, 2>::value)) k_batch_update_n(const __grid_constant__ BatchArgs<real> A) {
  __shared__ __align__(16) KParams<real> sP;
  constexpr bool MIXED = sizeof(real) == 4;
  const BatchTile tile = A.t_upd[A.upd_first[N - 3] + blockIdx.x];
  load_params(&sP, A.P + tile.prob);
  update_body<2, N, Eq2, real, MIXED, DegShape<N, T>::TB>(sP, A.tb[N - 3], A.td[N - 3], tile.blk,
                                                           A.nblk_upd[tile.prob], true);
}

// End of the step of every problem after the update phase: one warp per
// problem (finish_step_warp; the update blocks only folded their rates into
// the problem's rate counters).
template <typename real>
__global__ void k_batch_finish(const __grid_constant__ BatchArgs<real> A) {
  finish_step_warp(A.P[blockIdx.x].b.ctl);
}

template <typename real, int T>
__global__ void __launch_bounds__(T, (sizeof(real) == 4 ? 4 : 3) * 256 / T) k_batch_face(const __grid_constant__ BatchArgs<real> A) {
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

// Wait (thread 0) until done[] reaches target, at most A.spin_limit polls of
// at least 64 ns; gives up early when another block has set the error flag.
// Returns false (for the whole block) when the wait failed.
template <typename real>
__device__ bool wait_count(const BatchArgs<real>& A, const unsigned* cnt, unsigned target, int* sflag) {
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned long long spins = 0;
    while (*reinterpret_cast<const volatile unsigned*>(cnt) < target) {
      if (*reinterpret_cast<volatile int*>(A.err) != 0) {
        ok = 0;
        break;
      }
      if (++spins > A.spin_limit) {
        atomicOr(A.err, 1);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    *sflag = ok;
  }
  __syncthreads();
  return *reinterpret_cast<volatile int*>(sflag) != 0;
}

// Publish cnt finished tiles of counter idx (every thread; no-op when cnt is 0).
__device__ __forceinline__ void publish(unsigned* done, int idx, unsigned& cnt) {
  if (cnt == 0u) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(done + idx, cnt);
  }
  cnt = 0u;
}

template <typename real, int T>
__global__ void __launch_bounds__(T, (FusedMinBlocks<real, T>::value)) k_batch_fused(const __grid_constant__ BatchArgs<real> A) {
  __shared__ __align__(16) KParams<real> sP;
  __shared__ unsigned sNext;
  __shared__ int sFlag;
  int cur = -1;
  const unsigned per_step = unsigned(A.n_el) + unsigned(A.n_face) + unsigned(A.n_upd);
  const unsigned total = per_step * unsigned(A.nsteps);
  const unsigned chunk = unsigned(A.tiles) * kFusedClaim;
  unsigned* done = A.queue + 1;  // [phase][prob]
  if (threadIdx.x == 0) sNext = atomicAdd(A.queue, chunk);
  __syncthreads();
  unsigned first = sNext;
  int ok_key = -1;          // the last wait that ended, and its target (counts only grow)
  unsigned ok_target = 0u;
  int pend_idx = 0;         // finished tiles of one (phase, problem) not yet published
  unsigned pend = 0u;
  while (first < total) {
    __syncthreads();  // every thread has read sNext
    // claim the next chunk now: its latency overlaps this chunk's work
    if (threadIdx.x == 0)
      sNext = *reinterpret_cast<volatile int*>(A.err) ? total : atomicAdd(A.queue, chunk);
    const unsigned end = first + chunk < total ? first + chunk : total;
    for (unsigned item = first; item < end; ++item) {
      const int s = int(item / per_step);
      const int r = int(item - unsigned(s) * per_step);
      const int phase = r < A.n_el ? 0 : (r < A.n_el + A.n_face ? 1 : 2);
      const int t = phase == 0 ? r : (phase == 1 ? r - A.n_el : r - A.n_el - A.n_face);
      const int prob = phase == 1 ? A.t_face[t].prob : (phase == 0 ? A.t_el[t].prob : A.t_upd[t].prob);
      // the work this item reads: the previous step's update (local phase),
      // this step's local phase (face phase), this step's face phase (update)
      const int dep = phase == 0 ? 2 : phase - 1;
      const unsigned per = unsigned(dep == 0 ? A.nblk_el[prob] : (dep == 1 ? A.nblk_face[prob] : A.nblk_upd[prob]));
      const unsigned target = per * unsigned(phase == 0 ? s : s + 1) + unsigned(A.phantom);
      const int key = dep * A.nprob + prob;
      if (key != ok_key || target > ok_target) {
        publish(done, pend_idx, pend);  // never wait while holding unpublished work
        if (!wait_count(A, done + key, target, &sFlag)) return;
        ok_key = key;
        ok_target = target;
      }
      if (phase == 1) face_tile<real>(A, &sP, t, cur);
      else if (phase == 0) el_tile<real, 0, T>(A, &sP, t, cur);
      else el_tile<real, 2, T>(A, &sP, t, cur);
      const int idx = phase * A.nprob + prob;
      if (idx != pend_idx) publish(done, pend_idx, pend);
      pend_idx = idx;
      ++pend;
    }
    publish(done, pend_idx, pend);
    __syncthreads();
    first = sNext;
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

// Dynamic shared memory of the one-degree phase kernels (whole elements only).
template <typename real, int N, int T>
size_t smem_local_n() {
  return Impl<2, N, Eq2, real, sizeof(real) == 4>::smem_local(DegShape<N, T>::EPB);
}
template <typename real, int N, int T>
size_t smem_update_n() {
  return Impl<2, N, Eq2, real, sizeof(real) == 4>::smem_update(DegShape<N, T>::EPB);
}

template <typename real, int T>
cudaError_t configure_t() {
  const int sm = (int)smem_for<real>(T);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_batch_local_n<real, 3, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_local_n<real, 3, T>())))
    return e;
  if ((e = cudaFuncSetAttribute(k_batch_local_n<real, 4, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_local_n<real, 4, T>())))
    return e;
  if ((e = cudaFuncSetAttribute(k_batch_update_n<real, 3, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_update_n<real, 3, T>())))
    return e;
  if ((e = cudaFuncSetAttribute(k_batch_update_n<real, 4, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_update_n<real, 4, T>())))
    return e;
  return cudaFuncSetAttribute(k_batch_fused<real, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

template <typename real, int T>
cudaError_t launch_phase_t(int phase, const BatchArgs<real>& A, cudaStream_t s) {
  if (phase == 0) {  // one launch per degree present
    if (A.el_count[0] > 0)
      k_batch_local_n<real, 3, T><<<A.el_count[0], DegShape<3, T>::TB, smem_local_n<real, 3, T>(), s>>>(A);
    if (A.el_count[1] > 0)
      k_batch_local_n<real, 4, T><<<A.el_count[1], DegShape<4, T>::TB, smem_local_n<real, 4, T>(), s>>>(A);
  } else if (phase == 1) {
    if (A.n_face > 0) k_batch_face<real, T><<<A.n_face, T, 0, s>>>(A);
  } else {
    if (A.upd_count[0] > 0)
      k_batch_update_n<real, 3, T><<<A.upd_count[0], DegShape<3, T>::TB, smem_update_n<real, 3, T>(), s>>>(A);
    if (A.upd_count[1] > 0)
      k_batch_update_n<real, 4, T><<<A.upd_count[1], DegShape<4, T>::TB, smem_update_n<real, 4, T>(), s>>>(A);
    k_batch_finish<real><<<A.nprob, 32, 0, s>>>(A);
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
  // the queue head and the per-(phase, problem) completion counts start at zero
  cudaError_t e = cudaMemsetAsync(A.queue, 0, (1 + 3 * (size_t)A.nprob) * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
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
  if (threads != 128 && threads != 256) return cudaErrorInvalidValue;
  // both sizes: the update phase may run in blocks of its own size
  cudaError_t e = fp32 ? configure_t<float, 128>() : configure_t<double, 128>();
  if (e == cudaSuccess) e = fp32 ? configure_t<float, 256>() : configure_t<double, 256>();
  return e;
}

cudaError_t batch_fused_max_blocks(int threads, bool fp32, int* blocks) {
  if (threads == 128) return fp32 ? max_blocks_t<float, 128>(blocks) : max_blocks_t<double, 128>(blocks);
  if (threads == 256) return fp32 ? max_blocks_t<float, 256>(blocks) : max_blocks_t<double, 256>(blocks);
  return cudaErrorInvalidValue;
}

cudaError_t batch_launch_phase(int threads, int phase, const void* args, bool fp32, cudaStream_t s) {
  if (fp32) {
    const BatchArgs<float>& A = *static_cast<const BatchArgs<float>*>(args);
    const int t = phase == 2 ? A.upd_threads : threads;
    if (t == 128) return launch_phase_t<float, 128>(phase, A, s);
    if (t == 256) return launch_phase_t<float, 256>(phase, A, s);
  } else {
    const BatchArgs<double>& A = *static_cast<const BatchArgs<double>*>(args);
    const int t = phase == 2 ? A.upd_threads : threads;
    if (t == 128) return launch_phase_t<double, 128>(phase, A, s);
    if (t == 256) return launch_phase_t<double, 256>(phase, A, s);
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
