// Host-side launchers of the step kernels, one KernelSet per (dimension,
// degree, equation, precision).  The host context only sees KernelSet.
#pragma once
#include "cr_kernels.cuh"

namespace crk {

struct KernelSet {
  int dim, degree, nvars, nodes, mixed;
  int launches_per_step;
  // params points at a KParams<double> (FP64) or KParams<float> (FP32_BULK)
  cudaError_t (*step)(const void* params, cudaStream_t s);
  cudaError_t (*launch[4])(const void* params, cudaStream_t s);  // local, face, update, finish
  const char* names[4];
  cudaError_t (*prologue)(const void* params, cudaStream_t s);
  cudaError_t (*split)(const void* params, const double* in, cudaStream_t s);  // FP64 -> state
  cudaError_t (*join)(const void* params, double* out, cudaStream_t s);        // state -> FP64
  cudaError_t (*means)(const void* params, double* out, cudaStream_t s);       // [M][Ne] FP64
  cudaError_t (*configure)();
};

template <int DIM, int N, class EQ, typename real, bool MIXED>
struct Impl {
  static constexpr int n = N + 1;
  static constexpr int NP = DIM == 2 ? n * n : n;
  static constexpr int M = EQ::M;
  static constexpr int NFN = DIM == 2 ? n : 1;
  // variables per node in the element kernel's shared arrays (VarPack pads FP32 to pairs)
  static constexpr int MV = (M + VarPack<real>::VL - 1) / VarPack<real>::VL * VarPack<real>::VL;

  // elements per block: about 256 threads per block (at least one element);
  // the FP32-bulk update kernel takes UpdateShape's (128 threads)
  static constexpr int EPB = BlockShape<NP>::EPB;

  static size_t smem_local(int epb) {
    return (((size_t)5 * MV * epb * NP * sizeof(real) + 15) & ~(size_t)15) + (size_t)epb * sizeof(double) +
           (size_t)4 * n * n * sizeof(real) + (size_t)epb * 4 * sizeof(int);
  }
  static constexpr int RW = 2 * M > 4 ? 2 * M : 4;
  static constexpr int MU = M > 2 ? M : 2;
  static size_t smem_update(int epb) {
    return ((size_t)(MU + RW) * epb * NP + 16 * (size_t)epb) * sizeof(double) +
           (size_t)epb * (NP + 1) * sizeof(float);
  }

  static cudaError_t configure() {
    cudaError_t err;
    err = cudaFuncSetAttribute(k_local<DIM, N, EQ, real, MIXED>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_local(EPB));
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(k_update<DIM, N, EQ, real, MIXED>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_update(EPB));
    if (err != cudaSuccess) return err;
    return cudaFuncSetAttribute(k_prologue<DIM, N, EQ, real, MIXED>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_update(EPB));
  }

  static cudaError_t launch_local(const void* pv, cudaStream_t s) {
    const KParams<real>& P = *static_cast<const KParams<real>*>(pv);
    const int grid = (P.m.ne + EPB - 1) / EPB;
    k_local<DIM, N, EQ, real, MIXED><<<grid, EPB * NP, smem_local(EPB), s>>>(P);
    return cudaGetLastError();
  }
  static cudaError_t launch_face(const void* pv, cudaStream_t s) {
    const KParams<real>& P = *static_cast<const KParams<real>*>(pv);
    const int nfaces = P.m.ny * P.m.nfx * NFN + (DIM == 2 ? P.m.nfy * P.m.nx * n : 0);
    k_face<DIM, N, EQ, real><<<(nfaces + 255) / 256, 256, 0, s>>>(P);
    return cudaGetLastError();
  }
  static cudaError_t launch_update(const void* pv, cudaStream_t s) {
    const KParams<real>& P = *static_cast<const KParams<real>*>(pv);
    constexpr int EU = UpdateShape<NP, MIXED>::EPB;
    const int grid = (P.m.ne + EU - 1) / EU;
    k_update<DIM, N, EQ, real, MIXED><<<grid, EU * NP, smem_update(EU), s>>>(P);
    return cudaGetLastError();
  }
  static cudaError_t launch_finish(const void* pv, cudaStream_t s) {
    const KParams<real>& P = *static_cast<const KParams<real>*>(pv);
    k_finish_step<<<1, 32, 0, s>>>(P.b.ctl);
    return cudaGetLastError();
  }
  static cudaError_t step(const void* pv, cudaStream_t s) {
    cudaError_t e = launch_local(pv, s);
    if (e == cudaSuccess) e = launch_face(pv, s);
    if (e == cudaSuccess) e = launch_update(pv, s);
    if (e == cudaSuccess) e = launch_finish(pv, s);
    return e;
  }

  static cudaError_t prologue(const void* pv, cudaStream_t s) {
    const KParams<real>& P = *static_cast<const KParams<real>*>(pv);
    const int grid = (P.m.ne + EPB - 1) / EPB;
    k_prologue<DIM, N, EQ, real, MIXED><<<grid, EPB * NP, smem_update(EPB), s>>>(P);
    return cudaGetLastError();
  }

  static cudaError_t split(const void* pv, const double* in, cudaStream_t s) {
    const KParams<real>& P = *static_cast<const KParams<real>*>(pv);
    const size_t nvals = (size_t)M * P.m.ne * NP;
    if constexpr (MIXED) {
      const int nthr = M * P.m.ne;
      k_split_state<DIM, N, M><<<(nthr + 255) / 256, 256, 0, s>>>(in, P.b.u, P.b.umean, P.b.umean_f,
                                                                 P.m.ne, P.td);
      return cudaGetLastError();
    } else {
      return cudaMemcpyAsync(P.b.u, in, nvals * sizeof(double), cudaMemcpyDefault, s);
    }
  }

  static cudaError_t join(const void* pv, double* out, cudaStream_t s) {
    const KParams<real>& P = *static_cast<const KParams<real>*>(pv);
    const size_t nvals = (size_t)M * P.m.ne * NP;
    if constexpr (MIXED) {
      k_join_state<NP><<<(int)((nvals + 255) / 256), 256, 0, s>>>(P.b.u, P.b.umean, out, (int)nvals);
      return cudaGetLastError();
    } else {
      return cudaMemcpyAsync(out, P.b.u, nvals * sizeof(double), cudaMemcpyDefault, s);
    }
  }

  static cudaError_t means(const void* pv, double* out, cudaStream_t s) {
    const KParams<real>& P = *static_cast<const KParams<real>*>(pv);
    if constexpr (MIXED) {
      return cudaMemcpyAsync(out, P.b.umean, (size_t)M * P.m.ne * sizeof(double), cudaMemcpyDefault, s);
    } else {
      const int nthr = M * P.m.ne;
      k_element_means<DIM, N, M><<<(nthr + 255) / 256, 256, 0, s>>>(P.b.u, out, P.m.ne, P.td);
      return cudaGetLastError();
    }
  }

  static const KernelSet* set() {
    static const KernelSet ks = {DIM, N, M, NP, MIXED ? 1 : 0, 4, &step,
                                 {&launch_local, &launch_face, &launch_update, &launch_finish},
                                 {"k_local", "k_face", "k_update", "k_finish_step"},
                                 &prologue, &split, &join, &means, &configure};
    return &ks;
  }
};

// Registries, one per translation unit (equation x dimension).
const KernelSet* kernels_linadv1d(int N, int mixed);
const KernelSet* kernels_linadv2d(int N, int mixed);
const KernelSet* kernels_euler1d(int N, int mixed);
const KernelSet* kernels_euler2d(int N, int mixed);
const KernelSet* kernels_tenmoment1d(int N, int mixed);
const KernelSet* kernels_tenmoment2d(int N, int mixed);
const KernelSet* kernels_burgers1d(int N, int mixed);
const KernelSet* kernels_varadv1d(int N, int mixed);
const KernelSet* kernels_euler1d_grav(int N, int mixed);
const KernelSet* kernels_euler2d_grav(int N, int mixed);

}  // namespace crk
