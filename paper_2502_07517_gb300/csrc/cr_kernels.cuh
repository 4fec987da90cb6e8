// The three kernels of one cRKFR step and the prologue kernel, templated on
// dimension, degree N, equation and arithmetic type.
//
//   k_local   one thread per solution point, EPB elements per block: the local
//             cRK stages (Sec. 3 eq. (crkfr1)), the time averages F, G, U, S
//             (eqs. (disc.avg.flux), (time.avg.sol), App. B), the EA face fluxes
//             (eq. (evaluate)), the MUSCL-Hancock subcell states and fluxes
//             (Sec. 4.2) and the partial update: everything of eq.
//             (blended.scheme) except the element-face numerical fluxes.
//   k_face    one thread per face node: D2 high-order flux (eqs. (numflux.general),
//             (D2)), low-order flux, blend (eq. (Fblend)) and the flux limiter
//             (Sec. 4.3) in FP64.
//   k_update  one thread per solution point: adds the face-flux terms, applies
//             the scaling limiter, evaluates the smoothness indicator of the new
//             state and the CFL rate for the next step (eq. (time.step.2d)).
//
// State layout [M][Ne][Np]; element-local data are staged in shared memory as
// [M][EPB][Np] so that consecutive threads touch consecutive words.
#pragma once
#include "cr_common.cuh"

namespace crk {

__device__ __forceinline__ int neighbour(const Mesh& m, int e, int f) {
  const int ix = e % m.nx, iy = e / m.nx;
  if (f == 0) return ix > 0 ? e - 1 : (m.bcx == 0 ? e + m.nx - 1 : -1);
  if (f == 1) return ix < m.nx - 1 ? e + 1 : (m.bcx == 0 ? e - m.nx + 1 : -1);
  if (f == 2) return iy > 0 ? e - m.nx : (m.bcy == 0 ? e + m.nx * (m.ny - 1) : -1);
  return iy < m.ny - 1 ? e + m.nx : (m.bcy == 0 ? e - m.nx * (m.ny - 1) : -1);
}

// minmod of three slopes: the one of smallest magnitude when all three share a
// nonzero sign, else 0.
__device__ __forceinline__ float minmod3(float a, float b, float c) {
  if (a > 0.0f && b > 0.0f && c > 0.0f) return fminf(a, fminf(b, c));
  if (a < 0.0f && b < 0.0f && c < 0.0f) return fmaxf(a, fmaxf(b, c));
  return 0.0f;
}
// FP64 version on the bit patterns (integer pipe; the FP64 pipe is the scarce
// unit): sign bits must agree and no magnitude may be zero; for finite numbers
// of one sign the order of the magnitude bits is the order of the magnitudes.
__device__ __forceinline__ double minmod3(double a, double b, double c) {
  const unsigned long long ia = (unsigned long long)__double_as_longlong(a);
  const unsigned long long ib = (unsigned long long)__double_as_longlong(b);
  const unsigned long long ic = (unsigned long long)__double_as_longlong(c);
  const unsigned long long mag = 0x7fffffffffffffffull;
  const unsigned long long ma = ia & mag, mb = ib & mag, mc = ic & mag;
  if (((ia ^ ib) | (ia ^ ic)) >> 63 || ma == 0ull || mb == 0ull || mc == 0ull) return 0.0;
  unsigned long long mm = ma < mb ? ma : mb;
  mm = mm < mc ? mm : mc;
  return __longlong_as_double((long long)(mm | (ia & ~mag)));
}

// All admissibility constraints P_k > 0, evaluated exactly (Sec. 2 eq. (uad.form)).
template <class EQ, typename real>
__device__ __forceinline__ bool admissible(const real* u, const Phys<real>& ph) {
  bool ok = true;
#pragma unroll
  for (int k = 0; k < EQ::K; ++k) ok = ok && (EQ::constraint(u, k, ph) > real(0));
  return ok;
}

// Rusanov flux, Sec. 2 eqs. (num.flux.fr), (rusanov.wave.speed), at position x
// along the normal (variable advection only).
template <class EQ, typename real>
__device__ __forceinline__ void rusanov(const real* uL, const real* uR, int dir, real* out,
                                        const Phys<real>& ph, real x = real(0)) {
  real fL[EQ::M], fR[EQ::M], sL, sR;
  flux_speed_at<EQ>(uL, dir, fL, &sL, ph, x);
  flux_speed_at<EQ>(uR, dir, fR, &sR, ph, x);
  const real lam = fmax(sL, sR);
#pragma unroll
  for (int v = 0; v < EQ::M; ++v)
    out[v] = real(0.5) * (fL[v] + fR[v]) - real(0.5) * lam * (uR[v] - uL[v]);
}

// HLLC flux of the Euler equations (the upwind flux for boundaries that mix
// inflow and outflow, Sec. 3.3), normal direction dir, from states UL, UR and
// fluxes FL, FR given separately (time averages at a boundary face).  Davis
// wave speeds S_L = min(v_L - c_L, v_R - c_R), S_R = max(v_L + c_L, v_R + c_R),
// contact speed S* and star states of the classical three-wave solver.
template <class EQ, typename real>
__device__ __forceinline__ void hllc(int dir, const real* UL, const real* UR, const real* FL,
                                     const real* FR, real* out, const Phys<real>& ph) {
  constexpr int M = EQ::M;
  const int mn = 1 + dir, E = M - 1;
  const real rl = UL[0], rr = UR[0], vl = UL[mn] / rl, vr = UR[mn] / rr;
  const real pl = EQ::constraint(UL, 1, ph), pr = EQ::constraint(UR, 1, ph);
  const real cl = sqrt_pos(ph.gamma * pl / rl), cr = sqrt_pos(ph.gamma * pr / rr);
  const real sl = fmin(vl - cl, vr - cr), sr = fmax(vl + cl, vr + cr);
  if (sl >= real(0)) {
#pragma unroll
    for (int v = 0; v < M; ++v) out[v] = FL[v];
    return;
  }
  if (sr <= real(0)) {
#pragma unroll
    for (int v = 0; v < M; ++v) out[v] = FR[v];
    return;
  }
  const real ss = (pr - pl + rl * vl * (sl - vl) - rr * vr * (sr - vr)) / (rl * (sl - vl) - rr * (sr - vr));
  const bool left = ss >= real(0);
  const real* U = left ? UL : UR;
  const real* F = left ? FL : FR;
  const real r = left ? rl : rr, vn = left ? vl : vr, p = left ? pl : pr, sk = left ? sl : sr;
  const real fac = r * (sk - vn) / (sk - ss);
  real us[M];
#pragma unroll
  for (int v = 0; v < M; ++v) us[v] = fac * U[v] / r;
  us[0] = fac;
  us[mn] = fac * ss;
  us[E] = fac * (U[E] / r + (ss - vn) * (ss + p / (r * (sk - vn))));
#pragma unroll
  for (int v = 0; v < M; ++v) out[v] = F[v] + sk * (us[v] - U[v]);
}

// Load variable v of node k of element e from the state (mean + fluctuation
// in FP32_BULK mode).
template <typename real, bool MIXED>
__device__ __forceinline__ real load_state(const Bufs<real>& b, int ne, int NP, int v, int e,
                                           int k) {
  const real x = b.u[((size_t)v * ne + e) * NP + k];
  if constexpr (MIXED) return b.umean_f[(size_t)v * ne + e] + x;
  return x;
}

// slot buffer index: field f (0 sigma, 1.. U, 1+M.. EA, 1+2M.. u*, 1+3M.. base)
__device__ __forceinline__ size_t slot_index(int f, int side, int e, int j, int nside, int ne,
                                             int nfn) {
  return (((size_t)f * nside + side) * ne + e) * nfn + j;
}

// Per-element reductions of W quantities per element over the element's
// threads: buf[(w * epb + el) * NP + k] holds node k's value, and the result
// lands in buf[(w * epb + el) * NP].  Called by every thread.  One thread per
// (quantity, element) folds the NP values in node order: the W * epb folds sit
// in the block's first warps, where a tree would make every warp issue each of
// its levels with a few lanes active and wait at a barrier per level.
template <int NP, int W, typename T, class Op>
__device__ __forceinline__ void elem_reduce(T* buf, int epb, int el, int k, Op op) {
  __syncthreads();
  for (int t = threadIdx.x; t < W * epb; t += blockDim.x) {
    T* b = buf + t * NP;  // t = w * epb + element
    T acc = b[0];
#pragma unroll
    for (int i = 1; i < NP; ++i) acc = op(acc, b[i]);
    b[0] = acc;
  }
  __syncthreads();
}

struct OpSum {
  template <typename T>
  __device__ T operator()(T a, T b) const { return a + b; }
};
struct OpMin {
  template <typename T>
  __device__ T operator()(T a, T b) const { return fmin(a, b); }
};

// ---------------------------------------------------------------------------
// Arithmetic over the M variables of a point.  In FP32 the variables go two at
// a time through Blackwell's packed FP32 instructions (FFMA2, FADD2, FMUL2: one
// instruction for two lanes, each lane rounded exactly like the scalar
// instruction), so the results equal those of the scalar loop bit for bit with
// half the issue slots; FP64 stays scalar.  The element kernel's shared-memory
// node arrays keep the two variables of a pair side by side in FP32
// (VarPack<float>::VL = 2, one 64-bit access per pair): variable v of node
// slot i sits at base[((v / VL) * stride + i) * VL + v % VL], so the groups of
// a node lie GS = VL * stride apart.
template <typename real> struct VarPack { static constexpr int VL = 1; };
template <> struct VarPack<float> { static constexpr int VL = 2; };

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// y = fma(a, x, z) per variable (y may alias x or z)
template <int M>
__device__ __forceinline__ void vfma(float (&y)[M], float a, const float (&x)[M], const float (&z)[M]) {
#pragma unroll
  for (int v = 0; v + 1 < M; v += 2) {
    const float2 r = __ffma2_rn(f2(a, a), f2(x[v], x[v + 1]), f2(z[v], z[v + 1]));
    y[v] = r.x;
    y[v + 1] = r.y;
  }
  if (M & 1) y[M - 1] = fmaf(a, x[M - 1], z[M - 1]);
}
template <int M>
__device__ __forceinline__ void vfma(double (&y)[M], double a, const double (&x)[M], const double (&z)[M]) {
#pragma unroll
  for (int v = 0; v < M; ++v) y[v] = fma(a, x[v], z[v]);
}
// y = fma(a, x, y) per variable
template <int M, typename real>
__device__ __forceinline__ void vfma(real (&y)[M], real a, const real (&x)[M]) {
  vfma(y, a, x, y);
}
// y = x - z per variable (as fma(z, -1, x): the same rounding as the subtraction)
template <int M>
__device__ __forceinline__ void vsub(float (&y)[M], const float (&x)[M], const float (&z)[M]) {
#pragma unroll
  for (int v = 0; v + 1 < M; v += 2) {
    const float2 r = __ffma2_rn(f2(z[v], z[v + 1]), f2(-1.0f, -1.0f), f2(x[v], x[v + 1]));
    y[v] = r.x;
    y[v + 1] = r.y;
  }
  if (M & 1) y[M - 1] = x[M - 1] - z[M - 1];
}
template <int M>
__device__ __forceinline__ void vsub(double (&y)[M], const double (&x)[M], const double (&z)[M]) {
#pragma unroll
  for (int v = 0; v < M; ++v) y[v] = x[v] - z[v];
}
// y = x * a per variable
template <int M>
__device__ __forceinline__ void vmul(float (&y)[M], const float (&x)[M], float a) {
#pragma unroll
  for (int v = 0; v + 1 < M; v += 2) {
    const float2 r = __fmul2_rn(f2(x[v], x[v + 1]), f2(a, a));
    y[v] = r.x;
    y[v + 1] = r.y;
  }
  if (M & 1) y[M - 1] = x[M - 1] * a;
}
template <int M>
__device__ __forceinline__ void vmul(double (&y)[M], const double (&x)[M], double a) {
#pragma unroll
  for (int v = 0; v < M; ++v) y[v] = x[v] * a;
}
// y = fma(a, (node values at p), y): p points at the node's first variable
template <int M, int GS>
__device__ __forceinline__ void vfma_sh(float (&y)[M], float a, const float* p) {
#pragma unroll
  for (int v = 0; v + 1 < M; v += 2) {
    const float2 x = *reinterpret_cast<const float2*>(p + (v / 2) * GS);
    const float2 r = __ffma2_rn(f2(a, a), x, f2(y[v], y[v + 1]));
    y[v] = r.x;
    y[v + 1] = r.y;
  }
  if (M & 1) y[M - 1] = fmaf(a, p[(M / 2) * GS], y[M - 1]);
}
template <int M, int GS>
__device__ __forceinline__ void vfma_sh(double (&y)[M], double a, const double* p) {
#pragma unroll
  for (int v = 0; v < M; ++v) y[v] = fma(a, p[v * GS], y[v]);
}
// node values at p -> x, and x -> node values at p
template <int M, int GS>
__device__ __forceinline__ void vld_sh(float (&x)[M], const float* p) {
#pragma unroll
  for (int v = 0; v + 1 < M; v += 2) {
    const float2 w = *reinterpret_cast<const float2*>(p + (v / 2) * GS);
    x[v] = w.x;
    x[v + 1] = w.y;
  }
  if (M & 1) x[M - 1] = p[(M / 2) * GS];
}
template <int M, int GS>
__device__ __forceinline__ void vld_sh(double (&x)[M], const double* p) {
#pragma unroll
  for (int v = 0; v < M; ++v) x[v] = p[v * GS];
}
template <int M, int GS>
__device__ __forceinline__ void vst_sh(float* p, const float (&x)[M]) {
#pragma unroll
  for (int v = 0; v + 1 < M; v += 2) *reinterpret_cast<float2*>(p + (v / 2) * GS) = f2(x[v], x[v + 1]);
  if (M & 1) p[(M / 2) * GS] = x[M - 1];
}
template <int M, int GS>
__device__ __forceinline__ void vst_sh(double* p, const double (&x)[M]) {
#pragma unroll
  for (int v = 0; v < M; ++v) p[v * GS] = x[v];
}

// Face-node slot gs of a block, the slots numbered across the block so that
// the threads left without one form whole idle warps (FP64 pipe time and
// issue slots are charged per warp instruction): element el of the block
// (gs / NSLOT), its side and node j along that face.
struct FaceSlot {
  int el, side, j;
};
template <int NSLOT, int NFN>
__device__ __forceinline__ FaceSlot face_slot(int gs) {
  FaceSlot f;
  f.el = gs / NSLOT;
  const int sl = gs - f.el * NSLOT;
  f.side = sl / NFN;
  f.j = sl - f.side * NFN;
  return f;
}

// ===========================================================================
// Body of k_local for block blk of a problem (the standalone kernel and the
// batched kernels of cr_batch.cu call it).  Threads past the block's last whole
// element form an invalid "ghost" slot, so any block size works.
template <int DIM, int N, class EQ, typename real, bool MIXED, int T>
__device__ __forceinline__ void local_body(const KParams<real>& P, const Tab<real>& tb,
                                           const int blk) {
  constexpr int n = N + 1;
  constexpr int NP = DIM == 2 ? n * n : n;
  constexpr int M = EQ::M;
  constexpr int S = Tableau<N>::S;
  constexpr int NSIDE = DIM == 2 ? 4 : 2;
  constexpr int NFN = DIM == 2 ? n : 1;
  constexpr int NSLOT = NSIDE * NFN;
  constexpr int SPT = (NSLOT + NP - 1) / NP;
  using TB = Tableau<N>;
  const Mesh& m = P.m;
  const Phys<real>& ph = P.ph;
  constexpr int epb = (T + NP - 1) / NP;  // element slots in shared memory
  constexpr int epr = T / NP;             // whole elements of the block
  const int tid = threadIdx.x;
  const int el = tid / NP, k = tid - el * NP;
  const int p = DIM == 2 ? k % n : k, q = DIM == 2 ? k / n : 0;
  const int e = blk * epr + el;
  const bool valid = el < epr && e < m.ne;
  const int ee = valid ? e : m.ne - 1;
  const int ix = ee % m.nx, iy = ee / m.nx;

  const double dtd = P.b.ctl->dt_step;
  if (!gt0(dtd)) return;  // (integer test: the FP64 pipe is the scarce unit)
  const real dt = sizeof(real) == 4 ? real(P.b.ctl->dt_step_f) : real(dtd);
  // position of the node along x, for a flux that depends on it (variable advection)
  constexpr bool XDEP = IsVarAdv<EQ>::value;
  const real xnode = XDEP ? real(m.x0 + (ix + double(tb.xi[p])) * m.dx) : real(0);

  extern __shared__ __align__(16) unsigned char smem_raw[];
  real* sh = reinterpret_cast<real*>(smem_raw);
  // node arrays [M / VL][epb][NP][VL] (VarPack: FP32 variable pairs side by side)
  constexpr int VL = VarPack<real>::VL;
  constexpr int MV = (M + VL - 1) / VL * VL;
  constexpr int stride = epb * NP;
  constexpr int GS = VL * stride;
  constexpr int arr = MV * stride;
  real* s0 = sh;
  real* sA = sh + arr;
  real* sB = sA + arr;
  real* sC = sB + arr;
  real* sD = sC + arr;
#define AT(base, v, node) base[(((v) / VL) * stride + el * NP + (node)) * VL + (v) % VL]
#define ATE(base, v, elx, node) base[(((v) / VL) * stride + (elx) * NP + (node)) * VL + (v) % VL]
#define ATP(base, node) (&AT(base, 0, node))
#define ATPE(base, elx, node) (&ATE(base, 0, elx, node))

  real un[M];
#pragma unroll
  for (int v = 0; v < M; ++v) un[v] = load_state<real, MIXED>(P.b, m.ne, NP, v, ee, k);
  vst_sh<M, GS>(ATP(s0, k), un);

  // blending coefficient alpha_e, smoothed with the face neighbours, broadcast
  // through shared memory.  FP64: the block's elements side by side in its
  // first threads (one FP64-pipe warp instruction per operation for the whole
  // block); FP32 bulk: thread 0 of each element (measured 2.5% faster there).
  double* sAlpha = reinterpret_cast<double*>(
      smem_raw + (((size_t)5 * MV * epb * NP * sizeof(real) + 15) & ~(size_t)15));
  // the element's face neighbours (-1: a boundary side) are kept in shared
  // memory for the MUSCL-Hancock halo as well (measured 2.3% faster FP32 bulk
  // k_local than every boundary node recomputing them)
  int* sNbr = reinterpret_cast<int*>(reinterpret_cast<real*>(sAlpha + epb) + 4 * n * n);  // [epb][4]
  auto smooth_alpha = [&](int e2, int eg, bool v2) {
    int nbs[NSIDE];
#pragma unroll
    for (int f = 0; f < NSIDE; ++f) {
      nbs[f] = neighbour(m, eg, f);
      sNbr[e2 * 4 + f] = nbs[f];
    }
    if constexpr (MIXED) {
      // from the FP32 copies: max and halving commute with the rounding to FP32,
      // so this is the FP32 value of the FP64 smoothing, without FP64 work
      float al = 0.0f;
      double ald = 0.0;
      if (m.alpha_mode == 1) {
        ald = m.alpha_fixed;
        al = float(ald);
      } else if (m.limiter & kLimBlend) {
        al = P.b.alpha_raw_f[eg];
#pragma unroll
        for (int f = 0; f < NSIDE; ++f)
          if (nbs[f] >= 0) al = fmaxf(al, 0.5f * P.b.alpha_raw_f[nbs[f]]);
        ald = double(al);
      }
      reinterpret_cast<real*>(sAlpha)[e2] = al;
      if (v2) P.b.alpha[eg] = ald;
    } else {
      double al = 0.0;
      if (m.alpha_mode == 1) {
        al = m.alpha_fixed;
      } else if (m.limiter & kLimBlend) {
        al = P.b.alpha_raw[eg];
#pragma unroll
        for (int f = 0; f < NSIDE; ++f)
          if (nbs[f] >= 0) al = fmax(al, 0.5 * P.b.alpha_raw[nbs[f]]);
      }
      reinterpret_cast<real*>(sAlpha)[e2] = real(al);
      if (v2) P.b.alpha[eg] = al;
    }
  };
  if constexpr (MIXED) {
    if (k == 0) smooth_alpha(el, ee, valid);
  } else {
    for (int e2 = tid; e2 < epb; e2 += T) {
      const int eg0 = blk * epr + e2;
      const bool v2 = e2 < epr && eg0 < m.ne;
      smooth_alpha(e2, v2 ? eg0 : m.ne - 1, v2);
    }
  }
  // the scaled differentiation matrices, read by row with a per-thread row
  // index: from shared memory (measured 5% faster than from the kernel
  // parameters, where such an index makes a divergent constant-bank load)
  real* sDx = reinterpret_cast<real*>(sAlpha + epb);
  real* sDy = sDx + n * n;
  real* sDtx = sDy + n * n;
  real* sDty = sDtx + n * n;
  for (int t = tid; t < n * n; t += T) {
    sDx[t] = P.ds.Dx[t];
    sDy[t] = P.ds.Dy[t];
    sDtx[t] = P.ds.Dtx[t];
    sDty[t] = P.ds.Dty[t];
  }
  __syncthreads();
  const real alpha = reinterpret_cast<real*>(sAlpha)[el];
  const bool blend = (m.limiter & kLimBlend) || m.alpha_mode == 1;
  const bool need_lo = blend || (m.limiter & kLimFlux);
  const real a = blend ? alpha : real(0);

  // source: grad W at this node (ten-moment; time independent) or gravity (Euler)
  const bool has_src = (EQ::M == 6 && m.source == 1) || (HasGravity<EQ>::value && m.source == 2);
  real dWx = real(0), dWy = real(0);
  if (HasGravity<EQ>::value && has_src) {
    dWx = real(m.grav[0]);
    dWy = real(DIM == 2 ? m.grav[1] : 0.0);
  } else if (has_src) {
    const double x = m.x0 + (ix + double(tb.xi[p])) * m.dx;
    const double y = DIM == 2 ? m.y0 + (iy + double(tb.xi[q])) * m.dy : 0.0;
    source_grad<DIM, real>(m, real(x - m.src_cx), real(DIM == 2 ? y - m.src_cy : 0.0), &dWx, &dWy);
  }

  // ---------------- local cRK stages -----------------------------------
  real Lst[S > 1 ? S - 1 : 1][M];
  real Fa[M], Ga[M], Ua[M];
  real ea[SPT][M];
#pragma unroll
  for (int v = 0; v < M; ++v) {
    Fa[v] = Ga[v] = Ua[v] = real(0);
#pragma unroll
    for (int mm = 0; mm < SPT; ++mm) ea[mm][v] = real(0);
  }
  const real invdx = ph.invdx, invdy = ph.invdy;

#pragma unroll
  for (int i = 0; i < S; ++i) {
    // u^(i) = u^n - dt sum_j a_ij L_j; the arithmetic over the variables goes
    // through the v* helpers (FP32: two variables per instruction)
    real ui[M];
#pragma unroll
    for (int v = 0; v < M; ++v) ui[v] = un[v];
#pragma unroll
    for (int j = 0; j < i; ++j)
      if (TB::a(i, j) != 0.0) vfma(ui, -(dt * real(TB::a(i, j))), Lst[j]);
    real f[M], g[M];
    if (DIM == 2) EQ::flux_xy(ui, f, g, ph);
    else flux_at<EQ>(ui, 0, f, ph, xnode);
    if (TB::b(i) != 0.0) {
      const real bi = real(TB::b(i));
      vfma(Fa, bi, f);
      if (DIM == 2) vfma(Ga, bi, g);
      vfma(Ua, bi, ui);
    }
    vst_sh<M, GS>(ATP(sA, k), ui);
    vst_sh<M, GS>(ATP(sB, k), f);
    if (DIM == 2) vst_sh<M, GS>(ATP(sC, k), g);
    __syncthreads();
    if (i < S - 1) {
      real h[M];  // (D f)/dx + (D g)/dy as one chain per variable
#pragma unroll
      for (int v = 0; v < M; ++v) h[v] = real(0);
#pragma unroll
      for (int r = 0; r < n; ++r) vfma_sh<M, GS>(h, sDx[p * n + r], ATP(sB, r + n * q));
      if (DIM == 2) {
#pragma unroll
        for (int r = 0; r < n; ++r) vfma_sh<M, GS>(h, sDy[q * n + r], ATP(sC, p + n * r));
      }
#pragma unroll
      for (int v = 0; v < M; ++v) Lst[i < S - 1 ? i : 0][v] = h[v];
      if (has_src) {  // the stage's source, from its node value still in shared memory
        real us[M], s[M];
        vld_sh<M, GS>(us, ATP(sA, k));
        source_eval<EQ>(us, dWx, dWy, s);
#pragma unroll
        for (int v = 0; v < M; ++v) Lst[i < S - 1 ? i : 0][v] -= s[v];
      }
    }
    if (TB::b(i) != 0.0) {
      const real bi = real(TB::b(i));
#pragma unroll
      for (int mm = 0; mm < SPT; ++mm) {
        const FaceSlot fs = face_slot<NSLOT, NFN>(tid + mm * T);
        if (fs.el < epr) {
          const int side = fs.side, j = fs.j;
          real ut[M], fn[M];
#pragma unroll
          for (int v = 0; v < M; ++v) ut[v] = real(0);
#pragma unroll
          for (int r = 0; r < n; ++r) {
            const real l = (side & 1) ? tb.l1[r] : tb.l0[r];
            vfma_sh<M, GS>(ut, l, ATPE(sA, fs.el, side < 2 ? r + n * j : j + n * r));
          }
          const int eg = blk * epr + fs.el;
          if (m.dissipation == 2 && eg < m.ne) {  // D-CSX: the stage trace, for the face kernel
#pragma unroll
            for (int v = 0; v < M; ++v)
              P.b.slot[slot_index(1 + 4 * M + i * M + v, side, eg, j, NSIDE, m.ne, NFN)] = ut[v];
          }
          if (m.central == 0) {  // EA, eq. (evaluate)
            flux_at<EQ>(ut, side >> 1, fn, ph,
                        XDEP ? real(m.x0 + (min(eg, m.ne - 1) % m.nx + side) * m.dx) : real(0));
            vfma(ea[mm], bi, fn);
          }
        }
      }
    }
    __syncthreads();
  }

  // ---------------- time averages: high-order volume part, face data ----
  vst_sh<M, GS>(ATP(sA, k), Ua);
  vst_sh<M, GS>(ATP(sB, k), Fa);
  if (DIM == 2) vst_sh<M, GS>(ATP(sC, k), Ga);
  __syncthreads();
  real HO[M];
#pragma unroll
  for (int v = 0; v < M; ++v) HO[v] = real(0);
#pragma unroll
  for (int r = 0; r < n; ++r) vfma_sh<M, GS>(HO, sDtx[p * n + r], ATP(sB, r + n * q));
  if (DIM == 2) {
#pragma unroll
    for (int r = 0; r < n; ++r) vfma_sh<M, GS>(HO, sDty[q * n + r], ATP(sC, p + n * r));
  }
  // time-averaged source S = sum_i b_i s(u^(i)) (App. B eq. (crkfr.source)):
  // both sources are linear in u (the ten-moment one for fixed grad W), so it
  // equals s(U) of the time-averaged solution.  HO becomes the high-order part
  // of the update, u^n - dt (1 - a) HO + dt S (the low-order part follows).
  real Sa[M];
#pragma unroll
  for (int v = 0; v < M; ++v) Sa[v] = real(0);
  if (has_src) {
    real us[M];
    vld_sh<M, GS>(us, ATP(sA, k));
    source_eval<EQ>(us, dWx, dWy, Sa);
  }
  const real dho = dt * (real(1) - a);  // per-thread constants, one rounding each
  vfma(HO, -dho, HO, un);
  if (has_src) vfma(HO, dt, Sa);
#pragma unroll
  for (int mm = 0; mm < SPT; ++mm) {
    const FaceSlot fs = face_slot<NSLOT, NFN>(tid + mm * T);
    const int eg = blk * epr + fs.el;
    if (fs.el < epr && eg < m.ne) {
      const int side = fs.side, j = fs.j;
      // slot 1..M: the trace the dissipation jumps over (U for D2, u^n for D1);
      // slot 1+M..: the central part (EA average, or for AE the trace of the
      // time-averaged flux F (x faces) or G (y faces), eq. (extrapolate))
      real Ut[M], ut[M], Ft[M];
#pragma unroll
      for (int v = 0; v < M; ++v) Ut[v] = ut[v] = Ft[v] = real(0);
#pragma unroll
      for (int r = 0; r < n; ++r) {
        const real l = (side & 1) ? tb.l1[r] : tb.l0[r];
        const int node = side < 2 ? r + n * j : j + n * r;
        vfma_sh<M, GS>(Ut, l, ATPE(sA, fs.el, node));
        vfma_sh<M, GS>(ut, l, ATPE(s0, fs.el, node));
        if (m.central == 1) vfma_sh<M, GS>(Ft, l, side < 2 ? ATPE(sB, fs.el, node) : ATPE(sC, fs.el, node));
      }
      real* sl_out = P.b.slot;
      sl_out[slot_index(0, side, eg, j, NSIDE, m.ne, NFN)] =
          speed_at<EQ>(ut, side >> 1, ph, XDEP ? real(m.x0 + (eg % m.nx + side) * m.dx) : real(0));
#pragma unroll
      for (int v = 0; v < M; ++v) {
        sl_out[slot_index(1 + v, side, eg, j, NSIDE, m.ne, NFN)] = m.dissipation == 1 ? ut[v] : Ut[v];
        sl_out[slot_index(1 + M + v, side, eg, j, NSIDE, m.ne, NFN)] =
            m.central == 1 ? Ft[v] : ea[mm][v];
      }
    }
  }
  if constexpr (MIXED) {
    // source contribution to the FP64 element mean, sum_k W_k S_k (per-element
    // sum; has_src is the same for the whole block)
    if (has_src) {
      __syncthreads();
      const real W = DIM == 2 ? tb.w[p] * tb.w[q] : tb.w[p];
#pragma unroll
      for (int v = 0; v < M; ++v) sA[v * stride + el * NP + k] = W * Sa[v];  // elem_reduce's layout
      elem_reduce<NP, M>(sA, epb, el, k, OpSum());
      for (int v = k; valid && v < M; v += NP)
        P.b.smean[(size_t)v * m.ne + e] = double(sA[v * stride + el * NP]);
    } else {
      for (int v = k; valid && v < M; v += NP) P.b.smean[(size_t)v * m.ne + e] = 0.0;
    }
  }
  __syncthreads();

  // ---------------- MUSCL-Hancock / first-order subcells -----------------
  real LO[M];
#pragma unroll
  for (int v = 0; v < M; ++v) LO[v] = real(0);
  if (need_lo) {
    real xm[M], xp[M], ym[M], yp[M];
#pragma unroll
    for (int v = 0; v < M; ++v) xm[v] = xp[v] = ym[v] = yp[v] = un[v];
    if (m.limiter & kLimMH) {
      const real beta = real(2) - alpha;
      // one-sided slopes scaled by beta (per-thread constants)
      const real bmx = beta * tb.ihm[p], bpx = beta * tb.ihp[p];
      const real bmy = DIM == 2 ? beta * tb.ihm[q] : real(0), bpy = DIM == 2 ? beta * tb.ihp[q] : real(0);
      real um[M], up[M], sx[M], sy[M];
      // x-line neighbours: the neighbour element's node across a face; at a
      // boundary the ghost node of that side: the own node (outflow), its
      // reflection (wall, normal momentum reversed) or the given state
      // (Dirichlet, inflow)
      const int nbL = p == 0 ? sNbr[el * 4 + 0] : -1;
      const int nbR = p == N ? sNbr[el * 4 + 1] : -1;
      const int sgx = p == 0 ? 0 : 1;
      const int bgx = m.bcs[sgx];
      real gvx[M];  // the given state at t^n (Dirichlet, inflow)
#pragma unroll
      for (int v = 0; v < M; ++v) gvx[v] = un[v];
      if (bgx == kBcDirichlet || bgx == kBcInflow) ghost_at<M>(m, sgx, P.b.ctl->t, gvx);
#pragma unroll
      for (int v = 0; v < M; ++v) {
        const real gx = bgx == kBcWall ? (v == 1 ? -un[v] : un[v]) : gvx[v];
        um[v] = p > 0 ? AT(s0, v, k - 1)
                      : (nbL >= 0 ? load_state<real, MIXED>(P.b, m.ne, NP, v, nbL, N + n * q) : gx);
        up[v] = p < N ? AT(s0, v, k + 1)
                      : (nbR >= 0 ? load_state<real, MIXED>(P.b, m.ne, NP, v, nbR, n * q) : gx);
      }
      // minmod of the scaled one-sided and central differences
      auto slopes = [&](real (&sl)[M], real b_m, real b_c, real b_p) {
        real d1[M], d2[M], d3[M];
        vsub(d1, un, um);
        vsub(d2, up, um);
        vsub(d3, up, un);
        vmul(d1, d1, b_m);
        vmul(d2, d2, b_c);
        vmul(d3, d3, b_p);
#pragma unroll
        for (int v = 0; v < M; ++v) sl[v] = minmod3(d1[v], d2[v], d3[v]);
      };
      slopes(sx, bmx, tb.ihc[p], bpx);
#pragma unroll
      for (int v = 0; v < M; ++v) sy[v] = real(0);
      if (DIM == 2) {
        const int nbB = q == 0 ? sNbr[el * 4 + 2] : -1;
        const int nbT = q == N ? sNbr[el * 4 + 3] : -1;
        const int sgy = q == 0 ? 2 : 3;
        const int bgy = m.bcs[sgy];
        real gvy[M];
#pragma unroll
        for (int v = 0; v < M; ++v) gvy[v] = un[v];
        if (bgy == kBcDirichlet || bgy == kBcInflow) ghost_at<M>(m, sgy, P.b.ctl->t, gvy);
#pragma unroll
        for (int v = 0; v < M; ++v) {
          const real gy = bgy == kBcWall ? (v == 2 ? -un[v] : un[v]) : gvy[v];
          um[v] = q > 0 ? AT(s0, v, k - n)
                        : (nbB >= 0 ? load_state<real, MIXED>(P.b, m.ne, NP, v, nbB, p + n * N) : gy);
          up[v] = q < N ? AT(s0, v, k + n)
                        : (nbT >= 0 ? load_state<real, MIXED>(P.b, m.ne, NP, v, nbT, p) : gy);
        }
        slopes(sy, bmy, tb.ihc[q], bpy);
      }
      real fxm[M], fxp[M], fym[M], fyp[M], Fm[M], Fp[M], Gm[M], Gp[M];
      vfma(fxm, tb.dm[p], sx, un);
      vfma(fxp, tb.dp[p], sx, un);
      vfma(fym, tb.dm[q], sy, un);
      vfma(fyp, tb.dp[q], sy, un);
      flux_at<EQ>(fxm, 0, Fm, ph, XDEP ? real(m.x0 + (ix + double(tb.xs[p])) * m.dx) : real(0));
      flux_at<EQ>(fxp, 0, Fp, ph, XDEP ? real(m.x0 + (ix + double(tb.xs[p + 1])) * m.dx) : real(0));
      if (DIM == 2) {
        EQ::flux(fym, 1, Gm, ph);
        EQ::flux(fyp, 1, Gp, ph);
      }
      real ex[M], exm[M], exp_[M], eym[M], eyp[M];
      const real hx = real(0.5) * dt * (tb.invw[p] * invdx);
      const real hy = DIM == 2 ? real(0.5) * dt * (tb.invw[q] * invdy) : real(0);
      vsub(ex, Fp, Fm);
      vmul(ex, ex, hx);
      if (DIM == 2) {
        real dg[M];
        vsub(dg, Gp, Gm);
        vfma(ex, hy, dg);
      }
      vsub(exm, fxm, ex);
      vsub(exp_, fxp, ex);
      vsub(eym, fym, ex);
      vsub(eyp, fyp, ex);
      bool ok = EQ::admissible_fast(fxm, ph) && EQ::admissible_fast(fxp, ph) &&
                EQ::admissible_fast(exm, ph) && EQ::admissible_fast(exp_, ph);
      if (DIM == 2)
        ok = ok && EQ::admissible_fast(fym, ph) && EQ::admissible_fast(fyp, ph) &&
             EQ::admissible_fast(eym, ph) && EQ::admissible_fast(eyp, ph);
      if (ok) {
#pragma unroll
        for (int v = 0; v < M; ++v) {
          xm[v] = exm[v];
          xp[v] = exp_[v];
          ym[v] = eym[v];
          yp[v] = eyp[v];
        }
      }
    }
    vst_sh<M, GS>(ATP(sA, k), xm);
    vst_sh<M, GS>(ATP(sB, k), xp);
    if (DIM == 2) {
      vst_sh<M, GS>(ATP(sC, k), ym);
      vst_sh<M, GS>(ATP(sD, k), yp);
    }
    __syncthreads();
    // subcell fluxes, numbered across the block (element r / NSF of the block:
    // its N * NFN x-subfaces, then in 2D its n * N y-subfaces) so that the
    // threads left without one form whole idle warps.  The flux of the
    // subface right of (above) node (p2, q2) reads that node's x+ (y+) state,
    // which no other flux reads, and overwrites it in place.
    constexpr int NSX = N * NFN, NSF = DIM == 2 ? 2 * N * n : N;
    for (int gs = tid; gs < epr * NSF; gs += T) {
      const int el2 = gs / NSF, r = gs - el2 * NSF;
      const bool isx = r < NSX;
      const int rr = isx ? r : r - NSX;
      const int p2 = isx ? rr % N : rr % n, q2 = isx ? rr / N : rr / n;
      const int node = p2 + n * q2;
      real* sL = isx ? sB : sD;
      const real* sR = isx ? sA : sC;
      const int nodeR = node + (isx ? 1 : n);
      real uL[M], uR[M], fr[M];
      vld_sh<M, GS>(uL, ATPE(sL, el2, node));
      vld_sh<M, GS>(uR, ATPE(sR, el2, nodeR));
      real xf = real(0);
      if constexpr (XDEP) {
        const int e2 = min(blk * epr + el2, m.ne - 1);
        xf = real(m.x0 + (e2 % m.nx + double(tb.xs[p2 + 1])) * m.dx);
      }
      rusanov<EQ>(uL, uR, isx ? 0 : 1, fr, ph, xf);
      vst_sh<M, GS>(ATPE(sL, el2, node), fr);
    }
    __syncthreads();
    // low-order residual of the interior subfaces (eq. (low.order.update))
    const real wx = tb.invw[p] * invdx, wy = DIM == 2 ? tb.invw[q] * invdy : real(0);
    {
      real fr[M], fl[M];  // subcell fluxes right of and left of the node (0 at the element faces)
#pragma unroll
      for (int v = 0; v < M; ++v) fr[v] = fl[v] = real(0);
      if (p < N) vld_sh<M, GS>(fr, ATP(sB, k));
      if (p > 0) vld_sh<M, GS>(fl, ATP(sB, k - 1));
      vsub(fr, fr, fl);
      vmul(LO, fr, wx);
      if (DIM == 2) {
#pragma unroll
        for (int v = 0; v < M; ++v) fr[v] = fl[v] = real(0);
        if (q < N) vld_sh<M, GS>(fr, ATP(sD, k));
        if (q > 0) vld_sh<M, GS>(fl, ATP(sD, k - n));
        vsub(fr, fr, fl);
        vfma(LO, wy, fr);
      }
    }
    // face-node data for the face kernel: evolved boundary state u* and the
    // candidate base of the flux limiter, u_b -+ c f_adj
#pragma unroll
    for (int mm = 0; mm < SPT; ++mm) {
      const FaceSlot fs = face_slot<NSLOT, NFN>(tid + mm * T);
      const int eg = blk * epr + fs.el;
      if (fs.el < epr && eg < m.ne) {
        const int side = fs.side, j = fs.j;
        int nb_node, adj_node;
        const real* ust;
        const real* adj;
        if (side == 0) { nb_node = n * j; adj_node = n * j; ust = sA; adj = sB; }
        else if (side == 1) { nb_node = N + n * j; adj_node = N - 1 + n * j; ust = sB; adj = sB; }
        else if (side == 2) { nb_node = j; adj_node = j; ust = sC; adj = sD; }
        else { nb_node = j + n * N; adj_node = j + n * (N - 1); ust = sD; adj = sD; }
        const real c = dt * ph.cflim[side] * ((side & 1) ? real(1) : real(-1));
        real us[M], ub[M], fa[M];
        vld_sh<M, GS>(us, ATPE(ust, fs.el, nb_node));
        vld_sh<M, GS>(ub, ATPE(s0, fs.el, nb_node));
        vld_sh<M, GS>(fa, ATPE(adj, fs.el, adj_node));
        vfma(ub, c, fa);
#pragma unroll
        for (int v = 0; v < M; ++v) {
          P.b.slot[slot_index(1 + 2 * M + v, side, eg, j, NSIDE, m.ne, NFN)] = us[v];
          P.b.slot[slot_index(1 + 3 * M + v, side, eg, j, NSIDE, m.ne, NFN)] = ub[v];
        }
      }
    }
  }

  // ---------------- partial update --------------------------------------
  if (valid) {
    const real dlo = dt * a;
    real val[M];
    vfma(val, -dlo, LO, HO);
#pragma unroll
    for (int v = 0; v < M; ++v) P.b.P[((size_t)v * m.ne + e) * NP + k] = val[v];
  }
#undef AT
#undef ATE
#undef ATP
#undef ATPE
}

// Resident blocks per SM the step kernels ask for (measured on GB300,
// 2D Euler N = 4, 512x512): FP32_BULK blocks are latency bound and gain from
// four 256-thread blocks per SM (64 registers; k_local 1.39 -> 1.05 ms,
// k_update 0.91 -> 0.60 ms); the FP64 k_local is bound by the FP64 pipe and
// gains 3% from two blocks (128 registers instead of 130); the FP64 k_update
// is bound by its barriers and gains from more resident blocks: 2.15 ms at
// one (106 registers), 1.91 at three (85), 1.75 at four (64).
template <bool MIXED> struct MinBlocks {
  static constexpr int local = MIXED ? 4 : 2, update = 4;
};

// Threads per block of the single-problem step kernels: the whole elements
// that fit in 256 threads (at least one); the FP32-bulk update kernel in 128
// (barrier bound: smaller blocks wait less at each barrier, 0.482 -> 0.411 ms
// at 512x512 N = 4; the FP64 update was slower so, 1.75 -> 1.88 ms).
template <int NP, int THREADS = 256> struct BlockShape {
  static constexpr int EPB = (THREADS / NP) > 0 ? (THREADS / NP) : 1;
  static constexpr int T = EPB * NP;
};
template <int NP, bool MIXED> using UpdateShape = BlockShape<NP, MIXED ? 128 : 256>;

template <int DIM, int N, class EQ, typename real, bool MIXED>
__global__ void __launch_bounds__(256, MinBlocks<MIXED>::local) k_local(const __grid_constant__ KParams<real> P) {
  local_body<DIM, N, EQ, real, MIXED, BlockShape<DIM == 2 ? (N + 1) * (N + 1) : N + 1>::T>(P, P.tb, blockIdx.x);
}

// ===========================================================================
template <int DIM, int N, class EQ, typename real>
__device__ __forceinline__ void face_body(const KParams<real>& P, const int blk) {
  constexpr int n = N + 1;
  constexpr int M = EQ::M;
  constexpr int NSIDE = DIM == 2 ? 4 : 2;
  constexpr int NFN = DIM == 2 ? n : 1;
  const Mesh& m = P.m;
  const double dtd = P.b.ctl->dt_step;
  if (!gt0(dtd)) return;  // (integer test: the FP64 pipe is the scarce unit)
  const int nX = m.ny * m.nfx * NFN;
  const int nY = DIM == 2 ? m.nfy * m.nx * n : 0;
  const int idx = blk * blockDim.x + threadIdx.x;
  if (idx >= nX + nY) return;
  int dir, j, eL, eR, fx_i = 0;
  size_t out_idx, vstride;
  real* out;
  if (idx < nX) {
    dir = 0;
    j = idx % NFN;
    const int r = idx / NFN, i = r % m.nfx, iy = r / m.nfx;
    fx_i = i;
    eR = i < m.nx ? i + m.nx * iy : -1;
    eL = i > 0 ? i - 1 + m.nx * iy : (m.bcx == 0 ? m.nx - 1 + m.nx * iy : -1);
    out = P.b.fx;
    out_idx = idx;
    vstride = (size_t)nX;
  } else {
    dir = 1;
    const int id2 = idx - nX;
    j = id2 % n;
    const int r = id2 / n, ix = r % m.nx, i = r / m.nx;
    eR = i < m.ny ? ix + m.nx * i : -1;
    eL = i > 0 ? ix + m.nx * (i - 1) : (m.bcy == 0 ? ix + m.nx * (m.ny - 1) : -1);
    out = P.b.fy;
    out_idx = id2;
    vstride = (size_t)nY;
  }
  const int sL = dir == 0 ? 1 : 3, sR = dir == 0 ? 0 : 2;
  // the face's position along x, for a flux that depends on it (variable advection)
  constexpr bool XDEP = IsVarAdv<EQ>::value;
  const real xf = XDEP && dir == 0 ? real(m.x0 + fx_i * m.dx) : real(0);
  const real* sl = P.b.slot;
  auto fld = [&](int f, int side, int e) { return sl[slot_index(f, side, e, j, NSIDE, m.ne, NFN)]; };

  real FHO[M], fLO[M];
  double alpha_f;
  const bool blend = (m.limiter & kLimBlend) || m.alpha_mode == 1;
  const bool need_lo = blend || (m.limiter & kLimFlux);
  if (eL >= 0 && eR >= 0) {
    if (m.dissipation == 2) {
      // D-CSX, eq. (dcsx): sum_i b_i lambda_i/2 (u^(i)+ - u^(i)-), lambda_i
      // from the stage traces of both sides
      real Dv[M];
#pragma unroll
      for (int v = 0; v < M; ++v) Dv[v] = real(0);
#pragma unroll
      for (int i = 0; i < Tableau<N>::S; ++i) {
        if (Tableau<N>::b(i) == 0.0) continue;
        real uL[M], uR[M];
#pragma unroll
        for (int v = 0; v < M; ++v) {
          uL[v] = fld(1 + 4 * M + i * M + v, sL, eL);
          uR[v] = fld(1 + 4 * M + i * M + v, sR, eR);
        }
        const real lam = fmax(speed_at<EQ>(uL, dir, P.ph, xf), speed_at<EQ>(uR, dir, P.ph, xf));
        const real bi = real(Tableau<N>::b(i));
#pragma unroll
        for (int v = 0; v < M; ++v) Dv[v] += bi * real(0.5) * lam * (uR[v] - uL[v]);
      }
#pragma unroll
      for (int v = 0; v < M; ++v)
        FHO[v] = real(0.5) * (fld(1 + M + v, sL, eL) + fld(1 + M + v, sR, eR)) - Dv[v];
    } else {  // D2 (slots 1..M hold U traces) or D1 (they hold u^n traces)
      const real lam = fmax(fld(0, sL, eL), fld(0, sR, eR));
#pragma unroll
      for (int v = 0; v < M; ++v)
        FHO[v] = real(0.5) * (fld(1 + M + v, sL, eL) + fld(1 + M + v, sR, eR)) -
                 real(0.5) * lam * (fld(1 + v, sR, eR) - fld(1 + v, sL, eL));
    }
    if (need_lo) {
      real uL[M], uR[M];
#pragma unroll
      for (int v = 0; v < M; ++v) {
        uL[v] = fld(1 + 2 * M + v, sL, eL);
        uR[v] = fld(1 + 2 * M + v, sR, eR);
      }
      rusanov<EQ>(uL, uR, dir, fLO, P.ph, xf);
    }
    alpha_f = 0.5 * (P.b.alpha[eL] + P.b.alpha[eR]);
  } else {
    // boundary face: the interior side (ei, slot side si) and the type of this side
    const int ei = eR >= 0 ? eR : eL;
    const int si = eR >= 0 ? sR : sL;
    const int side = eR >= 0 ? (dir == 0 ? 0 : 2) : (dir == 0 ? 1 : 3);
    const int bc = m.bcs[side];
    const bool given = bc == kBcDirichlet || bc == kBcInflow;
    // given ghost state at t^n, and at the stage times with the averages
    // U^- = sum_i b_i g_i, F^- = sum_i b_i f(g_i) (Sec. 3.3; g and f(g) when g
    // does not depend on time)
    const bool tdep = given && M == 1 && m.bcnt > 0;
    real gs[M], Ug[M], Fg[M], sg = real(0);
#pragma unroll
    for (int v = 0; v < M; ++v) gs[v] = Ug[v] = Fg[v] = real(0);
    if (given) {
      ghost_at<M>(m, side, P.b.ctl->t, gs);
      flux_speed_at<EQ>(gs, dir, Fg, &sg, P.ph, xf);
#pragma unroll
      for (int v = 0; v < M; ++v) Ug[v] = gs[v];
      if (tdep) {
#pragma unroll
        for (int v = 0; v < M; ++v) Ug[v] = Fg[v] = real(0);
#pragma unroll
        for (int i = 0; i < Tableau<N>::S; ++i) {
          real gi[M], fi[M];
          ghost_at<M>(m, side, P.b.ctl->t + tableau_c<N>(i) * dtd, gi);
          flux_at<EQ>(gi, dir, fi, P.ph, xf);
          const real bi = real(Tableau<N>::b(i));
#pragma unroll
          for (int v = 0; v < M; ++v) {
            Ug[v] += bi * gi[v];
            Fg[v] += bi * fi[v];
          }
        }
      }
    }
    if (IsEuler<EQ>::value && bc == kBcDirichlet && m.bcflux == 1) {
      // HLLC on the time-averaged ghost values (slots 1..M hold U: D1 is refused
      // with HLLC) and, for the low-order flux, on the evolved boundary state
      // against g(t^n)
      real Ui[M], Fi[M], us[M], fu[M], fg0[M];
#pragma unroll
      for (int v = 0; v < M; ++v) {
        Ui[v] = fld(1 + v, si, ei);
        Fi[v] = fld(1 + M + v, si, ei);
      }
      if (eR >= 0) hllc<EQ>(dir, Ug, Ui, Fg, Fi, FHO, P.ph);
      else hllc<EQ>(dir, Ui, Ug, Fi, Fg, FHO, P.ph);
      if (need_lo) {
#pragma unroll
        for (int v = 0; v < M; ++v) us[v] = fld(1 + 2 * M + v, si, ei);
        EQ::flux(us, dir, fu, P.ph);
        EQ::flux(gs, dir, fg0, P.ph);
        if (eR >= 0) hllc<EQ>(dir, gs, us, fg0, fu, fLO, P.ph);
        else hllc<EQ>(dir, us, gs, fu, fg0, fLO, P.ph);
      }
    } else if (bc == kBcWall || bc == kBcDirichlet) {
      // ghost values: wall, Sec. 3.3 eq. (reflect.time.avg): the interior u^n
      // trace and time-averaged solution with the normal momentum reversed, the
      // interior time-averaged flux with every other component reversed (the
      // reflection has the interior wave speed); Dirichlet: u^- = g(t^n),
      // U^- and F^- as above.  Then the scheme's flux as at an interior face.
      const bool wall = bc == kBcWall;
      real Dv[M];
      if (m.dissipation == 2) {  // D-CSX with ghost stage traces
#pragma unroll
        for (int v = 0; v < M; ++v) Dv[v] = real(0);
#pragma unroll
        for (int i = 0; i < Tableau<N>::S; ++i) {
          if (Tableau<N>::b(i) == 0.0) continue;
          real ui[M], gi[M];
#pragma unroll
          for (int v = 0; v < M; ++v) ui[v] = fld(1 + 4 * M + i * M + v, si, ei);
#pragma unroll
          for (int v = 0; v < M; ++v) gi[v] = gs[v];
          if (tdep) ghost_at<M>(m, side, P.b.ctl->t + tableau_c<N>(i) * dtd, gi);
          const real lam = wall ? speed_at<EQ>(ui, dir, P.ph, xf)
                                : fmax(speed_at<EQ>(ui, dir, P.ph, xf), speed_at<EQ>(gi, dir, P.ph, xf));
          const real bi = real(Tableau<N>::b(i));
#pragma unroll
          for (int v = 0; v < M; ++v) {
            const real ug = wall ? (v == 1 + dir ? -ui[v] : ui[v]) : gi[v];
            const real uL = eR >= 0 ? ug : ui[v], uR = eR >= 0 ? ui[v] : ug;
            Dv[v] += bi * real(0.5) * lam * (uR - uL);
          }
        }
      } else {
        const real lam = wall ? fld(0, si, ei) : fmax(fld(0, si, ei), sg);
#pragma unroll
        for (int v = 0; v < M; ++v) {
          const real Ui = fld(1 + v, si, ei);
          // the jump is of U (D2) or of u^n (D1): the ghost U^- or g(t^n)
          const real Ug_v = wall ? (v == 1 + dir ? -Ui : Ui) : (m.dissipation == 1 ? gs[v] : Ug[v]);
          const real UL = eR >= 0 ? Ug_v : Ui, UR = eR >= 0 ? Ui : Ug_v;
          Dv[v] = real(0.5) * lam * (UR - UL);
        }
      }
#pragma unroll
      for (int v = 0; v < M; ++v) {
        const real Fi = fld(1 + M + v, si, ei);
        const real Fgv = wall ? (v == 1 + dir ? Fi : -Fi) : Fg[v];
        const real FL = eR >= 0 ? Fgv : Fi, FR = eR >= 0 ? Fi : Fgv;
        FHO[v] = real(0.5) * (FL + FR) - Dv[v];
      }
      if (need_lo) {
        real us[M];
#pragma unroll
        for (int v = 0; v < M; ++v) us[v] = fld(1 + 2 * M + v, si, ei);
        if (wall) {
          // Rusanov between the evolved boundary state and its reflection; the
          // ghost flux is the interior flux reflected (one evaluation), so the
          // mass and energy components cancel exactly, as the reflection requires
          real fi[M], sp;
          EQ::flux_speed(us, dir, fi, &sp, P.ph);
#pragma unroll
          for (int v = 0; v < M; ++v) {
            const real fgv = v == 1 + dir ? fi[v] : -fi[v], ug = v == 1 + dir ? -us[v] : us[v];
            const real fl = eR >= 0 ? fgv : fi[v], fr = eR >= 0 ? fi[v] : fgv;
            const real ul = eR >= 0 ? ug : us[v], ur = eR >= 0 ? us[v] : ug;
            fLO[v] = real(0.5) * (fl + fr) - real(0.5) * sp * (ur - ul);
          }
        } else if (eR >= 0) {
          rusanov<EQ>(gs, us, dir, fLO, P.ph, xf);
        } else {
          rusanov<EQ>(us, gs, dir, fLO, P.ph, xf);
        }
      }
    } else if (bc == kBcInflow) {
      // fully inflow, Sec. 3.3: F = F^- (f(g) for a time-independent g), high
      // and low order
#pragma unroll
      for (int v = 0; v < M; ++v) FHO[v] = fLO[v] = Fg[v];
    } else {
      // fully outflow, Sec. 3.3: F = F^+ (the interior trace flux)
#pragma unroll
      for (int v = 0; v < M; ++v) FHO[v] = fld(1 + M + v, si, ei);
      if (need_lo) {
        real us[M];
#pragma unroll
        for (int v = 0; v < M; ++v) us[v] = fld(1 + 2 * M + v, si, ei);
        flux_at<EQ>(us, dir, fLO, P.ph, xf);
      }
    }
    alpha_f = P.b.alpha[ei];
  }
  // blended flux of eq. (Fblend) in the kernel's type
  const real af = real(alpha_f);
  real Fr[M];
#pragma unroll
  for (int v = 0; v < M; ++v) Fr[v] = blend ? (real(1) - af) * FHO[v] + af * fLO[v] : FHO[v];
  double theta = 1.0;
  bool limit = (m.limiter & kLimFlux) && EQ::K > 0;
  if (limit && sizeof(real) == 4) {
    // FP32 prescreen: when every candidate with the blended flux clears its
    // threshold 0.1 min P_k(candidate with f_LO) by a margin above FP32
    // rounding, the FP64 solve below would return theta = 1; skip it.
    const real dtf = real(P.b.ctl->dt_step_f);
    const real cLf = dtf * P.ph.cflim[dir == 0 ? 1 : 3], cRf = dtf * P.ph.cflim[dir == 0 ? 0 : 2];
    const real* Ff = Fr;
    bool safe = true;
#pragma unroll
    for (int kk = 0; kk < EQ::K; ++kk) {
      real lowL = real(0), lowR = real(0), hiL = real(0), hiR = real(0), sc = real(0);
      real cl[M], ch[M];
      if (eL >= 0) {
#pragma unroll
        for (int v = 0; v < M; ++v) {
          const real b = fld(1 + 3 * M + v, sL, eL);
          cl[v] = b - cLf * fLO[v];
          ch[v] = b - cLf * Ff[v];
          sc = fmax(sc, fabs(b));
        }
        lowL = EQ::constraint(cl, kk, P.ph);
        hiL = EQ::constraint(ch, kk, P.ph);
      }
      if (eR >= 0) {
#pragma unroll
        for (int v = 0; v < M; ++v) {
          const real b = fld(1 + 3 * M + v, sR, eR);
          cl[v] = b + cRf * fLO[v];
          ch[v] = b + cRf * Ff[v];
          sc = fmax(sc, fabs(b));
        }
        lowR = EQ::constraint(cl, kk, P.ph);
        hiR = EQ::constraint(ch, kk, P.ph);
      }
      const real margin = real(1e-4) * sc + real(1e-11);
      const real lowmin = eL >= 0 ? (eR >= 0 ? fmin(lowL, lowR) : lowL) : lowR;
      const real thr = real(0.1) * lowmin + margin;
      if (!(lowmin > real(20) * margin)) safe = false;
      if (eL >= 0 && !(hiL > thr)) safe = false;
      if (eR >= 0 && !(hiR > thr)) safe = false;
    }
    if (safe) limit = false;
  }
  if (limit) {
    const double cL = dtd * m.cflim[dir == 0 ? 1 : 3], cR = dtd * m.cflim[dir == 0 ? 0 : 2];
    double baseL[M], baseR[M], flo[M], F[M];
#pragma unroll
    for (int v = 0; v < M; ++v) F[v] = double(Fr[v]);
#pragma unroll
    for (int v = 0; v < M; ++v) {
      baseL[v] = eL >= 0 ? double(fld(1 + 3 * M + v, sL, eL)) : 0.0;
      baseR[v] = eR >= 0 ? double(fld(1 + 3 * M + v, sR, eR)) : 0.0;
      flo[v] = double(fLO[v]);
    }
#pragma unroll
    for (int kk = 0; kk < EQ::K; ++kk) {
      double cand[M], PlowL = 0.0, PlowR = 0.0, eps = INFINITY;
      if (eL >= 0) {
#pragma unroll
        for (int v = 0; v < M; ++v) cand[v] = baseL[v] - cL * flo[v];
        PlowL = EQ::constraint(cand, kk, P.phd);
        eps = fmin(eps, PlowL);
      }
      if (eR >= 0) {
#pragma unroll
        for (int v = 0; v < M; ++v) cand[v] = baseR[v] + cR * flo[v];
        PlowR = EQ::constraint(cand, kk, P.phd);
        eps = fmin(eps, PlowR);
      }
      eps *= 0.1;
      if (!(eps > 0.0)) {
        theta = 0.0;
        break;
      }
      double Ft[M], tk = 1.0;
#pragma unroll
      for (int v = 0; v < M; ++v) Ft[v] = theta * F[v] + (1.0 - theta) * flo[v];
      if (eL >= 0) {
#pragma unroll
        for (int v = 0; v < M; ++v) cand[v] = baseL[v] - cL * Ft[v];
        const double Pk = EQ::constraint(cand, kk, P.phd);
        if (Pk < eps) tk = fmin(tk, (PlowL - eps) / (PlowL - Pk));
      }
      if (eR >= 0) {
#pragma unroll
        for (int v = 0; v < M; ++v) cand[v] = baseR[v] + cR * Ft[v];
        const double Pk = EQ::constraint(cand, kk, P.phd);
        if (Pk < eps) tk = fmin(tk, (PlowR - eps) / (PlowR - Pk));
      }
      theta *= tk;
    }
#pragma unroll
    for (int v = 0; v < M; ++v) Fr[v] = real(theta * F[v] + (1.0 - theta) * flo[v]);
  }
#pragma unroll
  for (int v = 0; v < M; ++v) out[v * vstride + out_idx] = Fr[v];
}

// Resident blocks per SM of the face kernel (measured at 512x512 N = 4): FP32
// bulk 0.161 -> 0.108 ms at four (64 registers instead of 82), FP64 1.00 ->
// 0.99 ms at three (85 instead of 96).
template <int DIM, int N, class EQ, typename real>
__global__ void __launch_bounds__(256, sizeof(real) == 4 ? 4 : 3) k_face(const __grid_constant__ KParams<real> P) {
  face_body<DIM, N, EQ, real>(P, blockIdx.x);
}

// ===========================================================================
// Element-level helpers for k_update / k_prologue (one thread per node, EPB
// elements per block).  Per-element scalar work runs side by side in the
// block's first threads rather than on one lane per element (a warp
// instruction costs the FP64 pipe the same with 1 or 32 active lanes).

// Smoothness indicator of one element (the Hennemann et al. form, with T(N) and s
// of Mesh::T_ind, Mesh::s_ind):
// eps at the nodes in E[el*NP + k] -> Legendre modes -> energy fractions ->
// logistic alpha, returned on thread k = 0 of the element.  T is the
// arithmetic type (double in FP64 mode, float in FP32_BULK mode).
// With alpha mode 2 the learned network replaces the logistic map (see
// mlp_alpha); the indicator's alpha is the fallback when the network is not
// loaded or returns a non-finite value.  When feat is not null the network
// inputs of element e are written to feat[e * NP + k].
__device__ __forceinline__ float bf16_to_float(unsigned short h) {
  return __uint_as_float(((unsigned int)h) << 16);
}

constexpr int kMlpH = 32;

// Learned alpha: x_k = log10(e_k + 1e-10)/10 + 1 from the normalised modal
// energies e_k; two hidden layers of 32 ReLU units, sigmoid output; BF16
// weights, FP32 arithmetic.  Device weight layout (transposed by cr_mlp_load
// so that lane j of a warp reads entry j of 32 consecutive ones):
// W1T[NP][32], b1[32], W2T[32][32] (W2T[i][j] = W2[j][i]), b2[32], w3[32], b3.
// Every thread of the block calls this with its element's input x (thread k
// of element el); each full warp then evaluates whole elements, lane j being
// hidden unit j, and the output of element el is returned to all its threads.
// fbuf: shared memory for epb * (NP + 1) floats.
template <int NP>
__device__ float mlp_alpha(const unsigned short* __restrict__ w, float x, float* fbuf, int epb,
                           int el, int k) {
  float* X = fbuf;            // [epb][NP] inputs
  float* Y = fbuf + epb * NP; // [epb] outputs
  X[el * NP + k] = x;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned short* W1 = w;
  const unsigned short* B1 = W1 + NP * kMlpH;
  const unsigned short* W2 = B1 + kMlpH;
  const unsigned short* B2 = W2 + kMlpH * kMlpH;
  const unsigned short* W3 = B2 + kMlpH;
  const unsigned short* B3 = W3 + kMlpH;
  if (warp < nw) {  // full warps only (blockDim need not be a multiple of 32)
    // two elements per warp at a time: their dependent FMA chains interleave
    // (each element's arithmetic in the same order as alone)
    for (int e2 = warp; e2 < epb; e2 += 2 * nw) {
      const int e3 = e2 + nw < epb ? e2 + nw : e2;  // a second element, or e2 again
      const float* xa = X + e2 * NP;
      const float* xb = X + e3 * NP;
      float ha = bf16_to_float(B1[lane]), hb = ha;
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        const float wv = bf16_to_float(W1[i * kMlpH + lane]);
        ha = fmaf(wv, xa[i], ha);
        hb = fmaf(wv, xb[i], hb);
      }
      ha = fmaxf(ha, 0.0f);
      hb = fmaxf(hb, 0.0f);
      float aa = bf16_to_float(B2[lane]), ab = aa;
#pragma unroll
      for (int i = 0; i < kMlpH; ++i) {
        const float wv = bf16_to_float(W2[i * kMlpH + lane]);
        aa = fmaf(wv, __shfl_sync(0xffffffffu, ha, i), aa);
        ab = fmaf(wv, __shfl_sync(0xffffffffu, hb, i), ab);
      }
      const float w3 = bf16_to_float(W3[lane]);
      float za = w3 * fmaxf(aa, 0.0f), zb = w3 * fmaxf(ab, 0.0f);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        za += __shfl_xor_sync(0xffffffffu, za, o);
        zb += __shfl_xor_sync(0xffffffffu, zb, o);
      }
      if (lane == 0) {
        const float b3 = bf16_to_float(B3[0]);
        Y[e2] = 1.0f / (1.0f + expf(-(za + b3)));
        Y[e3] = 1.0f / (1.0f + expf(-(zb + b3)));
      }
    }
  }
  __syncthreads();
  return Y[el];
}

template <int DIM, int N, typename T>
__device__ T indicator_alpha(const Mesh& m, const Tab<T>& tb, T* E, T* Tm, T* red, int epb, int el,
                             int k, const int* mlp_flag, const unsigned short* mlp_w, float* fbuf,
                             float* feat, int e_out) {
  constexpr int n = N + 1;
  constexpr int NP = DIM == 2 ? n * n : n;
  T* Ee = E + el * NP;
  T* Te = Tm + el * NP;
  T mo;
  int i, j;
  if (DIM == 2) {
    i = k % n;
    j = k / n;
    T acc = T(0);
#pragma unroll
    for (int pp = 0; pp < n; ++pp) acc += tb.V[i * n + pp] * Ee[pp + n * j];
    Te[k] = acc;  // row transform, column j
    __syncthreads();
    mo = T(0);
#pragma unroll
    for (int q2 = 0; q2 < n; ++q2) mo += tb.V[j * n + q2] * Te[i + n * q2];
  } else {
    i = k;
    j = 0;
    mo = T(0);
#pragma unroll
    for (int pp = 0; pp < n; ++pp) mo += tb.V[k * n + pp] * Ee[pp];
  }
  const T e2 = mo * mo;
  const int mx = i > j ? i : j;
  // four sums: total, top (max index N), low (max index <= N-1), next-to-top (N-1)
  red[(0 * epb + el) * NP + k] = e2;
  red[(1 * epb + el) * NP + k] = mx == N ? e2 : T(0);
  red[(2 * epb + el) * NP + k] = mx <= N - 1 ? e2 : T(0);
  red[(3 * epb + el) * NP + k] = mx == N - 1 ? e2 : T(0);
  elem_reduce<NP, 4>(red, epb, el, k, OpSum());
  const T tot = red[(0 * epb + el) * NP];
  // the energy ratios and the logistic of every element of the block, side by
  // side in its first epb threads (one warp) rather than in thread 0 of each
  // element (one warp per element for this scalar work); the element's first
  // slot of Tm (free once the sums are done) carries the result back
  if (threadIdx.x < epb) {
    const int e2 = threadIdx.x;
    const T tot2 = red[(0 * epb + e2) * NP], top = red[(1 * epb + e2) * NP];
    const T low = red[(2 * epb + e2) * NP], top1 = red[(3 * epb + e2) * NP];
    const T r1 = tot2 > T(0) ? top / tot2 : T(0);
    const T r2 = (N >= 2 && low > T(0)) ? top1 / low : T(0);
    const T Ev = fmax(r1, r2);
    const T Tt = T(m.T_ind);
    T a2 = T(1) / (T(1) + exp(-T(m.s_ind) / Tt * (Ev - Tt)));
    if (a2 < T(1e-3)) a2 = T(0);
    if (a2 > T(1) - T(1e-3)) a2 = T(1);
    Tm[e2 * NP] = fmin(a2, T(1));
  }
  __syncthreads();
  T al = Tm[el * NP];
  if (m.alpha_mode == 2 || feat) {
    const float ek = tot > T(0) ? float(e2 / tot) : 0.0f;
    const float x = log10f(ek + 1e-10f) * 0.1f + 1.0f;
    if (feat && e_out >= 0) feat[(size_t)e_out * NP + k] = x;
    if (m.alpha_mode == 2 && mlp_flag && *mlp_flag) {
      const float y = mlp_alpha<NP>(mlp_w, x, fbuf, epb, el, k);
      if (k == 0 && isfinite(y)) {
        float ya = y;
        if (ya < 1e-3f) ya = 0.0f;
        if (ya > 1.0f - 1e-3f) ya = 1.0f;
        al = T(fminf(ya, 1.0f));
      }
    }
  }
  __syncthreads();  // red and Tm are reused by the caller
  return al;  // valid on k == 0 (on every thread of the element without a network)
}

// finish the step: block max of the CFL rate, last block publishes the rate,
// advances time when advance != 0, and resets the accumulators.
__device__ __forceinline__ void finish_block(TimeCtl* ctl, double block_rate, int advance,
                                             double dtd, int last_step, int nblk) {
  if (threadIdx.x == 0) {
    atomicMax(&ctl->rate_acc, (unsigned long long)__double_as_longlong(block_rate));
    __threadfence();
    const unsigned prev = atomicAdd(&ctl->blocks_done, 1u);
    if (prev == unsigned(nblk) - 1u) {
      __threadfence();
      const unsigned long long bits = atomicExch(&ctl->rate_acc, 0ull);
      ctl->rate_last = __longlong_as_double((long long)bits);
      ctl->blocks_done = 0;
      if (advance) {
        ctl->t = last_step ? ctl->t_final : ctl->t + dtd;
        ctl->steps += 1;
      }
      plan_step(ctl);
    }
  }
}

// End of a step of the single-problem path (one warp, launched after the
// update kernel): the maximum of the rate counters (rate_part) becomes the
// state's rate, the counters are cleared, time advances and the next step is
// planned.  The update blocks then only fold their rate into a counter (a
// reduction nobody waits for), where finish_block has every block wait for two
// round trips to one counter before it can retire (measured 11% of the
// FP32-bulk update kernel at 512x512 N = 4).
__device__ __forceinline__ void finish_step_warp(TimeCtl* ctl) {
  const double dtd = ctl->dt_step;
  if (!(dtd > 0.0)) return;  // no step was taken
  unsigned long long bits = 0ull;
  if (threadIdx.x < kRateParts) {
    unsigned long long* part = rate_part(ctl, threadIdx.x);
    bits = *part;
    *part = 0ull;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {  // bit patterns of non-negative doubles order as the values
    const unsigned long long other = __shfl_xor_sync(0xffffffffu, bits, o);
    bits = other > bits ? other : bits;
  }
  if (threadIdx.x != 0) return;
  ctl->rate_last = __longlong_as_double((long long)bits);
  ctl->t = ctl->last_step ? ctl->t_final : ctl->t + dtd;
  ctl->steps += 1;
  if (ctl->out) ctl->out_done = 1;
  plan_step(ctl);
}
static __global__ void k_finish_step(TimeCtl* ctl) { finish_step_warp(ctl); }

// CFL rate sigma_x(u_bar)/dx + sigma_y(u_bar)/dy of each element, block max,
// then finish_block (deferred: the block max goes into a rate counter, and
// finish_step_warp ends the step).  The block's elements are evaluated side
// by side by its first DIM * epb threads (one per element and direction) from the means in
// shared memory (means[e * mstride + v]; the elements of the block start at
// e_first, epr of them are whole).  A flux that depends on the position
// (variable advection, 1D) takes the largest sigma over the element's faces
// and solution points (xi: the nodes).  rbuf must not overlap means.
template <int DIM, int NP, class EQ, typename T>
__device__ __forceinline__ void rate_and_finish(const Mesh& m, const Phys<T>& ph, const T* means,
                                                int mstride, T* rbuf, int epb, int epr, int e_first,
                                                TimeCtl* ctl, int advance, double dtd, int last,
                                                int nblk, const T* xi, bool deferred = false) {
  if (threadIdx.x < DIM * epb) {
    const int e2 = threadIdx.x / DIM, kk = threadIdx.x - e2 * DIM;
    const int eg = e_first + e2;
    const bool ok = e2 < epr && eg < m.ne;
    T ub[EQ::M];
#pragma unroll
    for (int v = 0; v < EQ::M; ++v) ub[v] = means[e2 * mstride + v];
    T s;
    if constexpr (IsVarAdv<EQ>::value) {
      const double xe = m.x0 + ((ok ? eg : 0) % m.nx) * m.dx;
      s = fmax(speed_at<EQ>(ub, 0, ph, T(xe)), speed_at<EQ>(ub, 0, ph, T(xe + m.dx)));
      for (int pp = 0; pp < NP; ++pp) s = fmax(s, speed_at<EQ>(ub, 0, ph, T(xe + double(xi[pp]) * m.dx)));
    } else {
      s = EQ::speed(ub, kk, ph);
    }
    const T r = s * T(kk == 0 ? m.invdx : m.invdy);
    rbuf[e2 * 2 + kk] = ok ? r : T(0);
  }
  __syncthreads();
  // block max over the elements by the first warp (lane j: elements j, j + 32, ...),
  // then a shuffle tree: the maximum is the serial loop's, bit for bit, with one
  // dependent FP64 step per 32 elements instead of one per element
  double brate = 0.0;
  if (threadIdx.x < 32) {
    for (int j = threadIdx.x; j < epb; j += 32) {
      double r = double(rbuf[j * 2]);
      if (DIM == 2) r += double(rbuf[j * 2 + 1]);
      brate = fmax(brate, r);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) brate = fmax(brate, __shfl_xor_sync(0xffffffffu, brate, o));
  }
  if (deferred) {
    if (threadIdx.x == 0)
      atomicMax(rate_part(ctl, blockIdx.x % kRateParts), (unsigned long long)__double_as_longlong(brate));
    return;
  }
  finish_block(ctl, brate, advance, dtd, last, nblk);
}

// ===========================================================================
// k_update.  Shared memory (doubles): sU [MU][epb][NP] node values, sRed
// [RW][epb][NP] reduction buffer, sEl [epb][16] per-element values.
template <int DIM, int N, class EQ, typename real, bool MIXED, int T>
__device__ __forceinline__ void update_body(const KParams<real>& P, const Tab<real>& tb,
                                            const Tab<double>& td, const int blk, const int nblk,
                                            const bool deferred = false) {
  constexpr int n = N + 1;
  constexpr int NP = DIM == 2 ? n * n : n;
  constexpr int M = EQ::M;
  constexpr int NSIDE = DIM == 2 ? 4 : 2;
  constexpr int NFN = DIM == 2 ? n : 1;
  constexpr int NSLOT = NSIDE * NFN;
  constexpr int SPT = (NSLOT + NP - 1) / NP;
  constexpr int RW = 2 * M > 4 ? 2 * M : 4;
  constexpr int MU = M > 2 ? M : 2;
  const Mesh& m = P.m;
  const double dtd = P.b.ctl->dt_step;
  const int last_step = P.b.ctl->last_step;
  if (!gt0(dtd)) return;  // (integer test: the FP64 pipe is the scarce unit)
  constexpr int epb = (T + NP - 1) / NP;  // element slots in shared memory
  constexpr int epr = T / NP;             // whole elements of the block
  const int tid = threadIdx.x;
  const int el = tid / NP, k = tid - el * NP;
  const int p = DIM == 2 ? k % n : k, q = DIM == 2 ? k / n : 0;
  const int e = blk * epr + el;
  const bool valid = el < epr && e < m.ne;
  const int ee = valid ? e : m.ne - 1;
  const int ix = ee % m.nx, iy = ee / m.nx;
  constexpr int stride = epb * NP;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sU = reinterpret_cast<double*>(smem_raw);  // [MU][epb][NP]
  double* sRed = sU + MU * stride;                   // [RW][epb][NP]
  double* sEl = sRed + RW * stride;                  // [epb][16]
  float* sMlp = reinterpret_cast<float*>(sEl + 16 * epb);  // [epb][NP + 1] network scratch
  // per-element area: FP64 values at sEl[el*16 + 0..9] (0..3 limiter scalars, 4..9 the
  // FP64 mean); values in the kernel's type from double index 10 on: alpha at ER,
  // the FP32 mean copy at ER + 1 + v
  real* sElr = reinterpret_cast<real*>(sEl);
  constexpr int ES = int(16 * sizeof(double) / sizeof(real));
  constexpr int ER = int(10 * sizeof(double) / sizeof(real));
#define ATU(v, node) sU[(v) * stride + el * NP + (node)]
#define RED(w) sRed[((w) * epb + el) * NP + k]
#define RED0(w) sRed[((w) * epb + el) * NP]

  // ---- node update: partial update + element-face flux terms ------------
  const bool blend = (m.limiter & kLimBlend) || m.alpha_mode == 1;
  for (int e2 = tid; e2 < epb; e2 += T) {  // the block's elements side by side
    const int eg0 = blk * epr + e2;
    sElr[e2 * ES + ER] = real(P.b.alpha[(e2 < epr && eg0 < m.ne) ? eg0 : m.ne - 1]);
  }
  __syncthreads();
  const real a = blend ? sElr[el * ES + ER] : real(0);
  const real dt = MIXED ? real(P.b.ctl->dt_step_f) : real(dtd);
  const real one = real(1);
  const real invdx = P.ph.invdx, invdy = P.ph.invdy;
  const int ixR = m.bcx == 0 ? (ix + 1) % m.nx : ix + 1;
  const int iyT = DIM == 2 ? (m.bcy == 0 ? (iy + 1) % m.ny : iy + 1) : 0;
  const size_t nXf = (size_t)m.ny * m.nfx * NFN;
  const size_t nYf = DIM == 2 ? (size_t)m.nfy * m.nx * n : 0;
  // correction weights of the face fluxes, dt/dx and dt/dy folded in
  const real sx = dt * invdx, sy = DIM == 2 ? dt * invdy : real(0);
  const real cRx = sx * ((one - a) * tb.gR[p] + (p == N ? a * tb.invw[N] : real(0)));
  const real cLx = sx * ((one - a) * tb.gL[p] - (p == 0 ? a * tb.invw[0] : real(0)));
  const real cRy = DIM == 2 ? sy * ((one - a) * tb.gR[q] + (q == N ? a * tb.invw[N] : real(0))) : real(0);
  const real cLy = DIM == 2 ? sy * ((one - a) * tb.gL[q] - (q == 0 ? a * tb.invw[0] : real(0))) : real(0);
  const real W = DIM == 2 ? tb.w[p] * tb.w[q] : tb.w[p];
  real val[M];
#pragma unroll
  for (int v = 0; v < M; ++v) {
    const real FxL = P.b.fx[v * nXf + ((size_t)iy * m.nfx + ix) * NFN + q];
    const real FxR = P.b.fx[v * nXf + ((size_t)iy * m.nfx + ixR) * NFN + q];
    real x = P.b.P[((size_t)v * m.ne + ee) * NP + k] - FxR * cRx - FxL * cLx;
    if (DIM == 2) {
      const real GB = P.b.fy[v * nYf + ((size_t)iy * m.nx + ix) * n + p];
      const real GT = P.b.fy[v * nYf + ((size_t)iyT * m.nx + ix) * n + p];
      x = x - GT * cRy - GB * cLy;
    }
    val[v] = x;
  }
  real m32[M];
  double ubar[M];
  if constexpr (MIXED) {
    // FP32 mean of the nodal update (re-centring), per-element sum
    real* fRed = reinterpret_cast<real*>(sRed);
#pragma unroll
    for (int v = 0; v < M; ++v) fRed[(v * epb + el) * NP + k] = W * val[v];
    // element-face flux integrals sum_j w_j F_j in FP32, in a fixed order, so
    // that the two elements of a face obtain the same value (exact telescoping
    // of the FP64 mean update)
    real* fI = reinterpret_cast<real*>(sU);  // [epb][NSIDE * M]
    for (int t = k; t < NSIDE * M; t += NP) {
      const int side = t / M, v = t - side * M;
      real acc = real(0);
      if (side < 2) {
        const int fxi = side == 0 ? ix : ixR;
#pragma unroll
        for (int j = 0; j < NFN; ++j) {
          const real fv = P.b.fx[v * nXf + ((size_t)iy * m.nfx + fxi) * NFN + j];
          acc += DIM == 2 ? tb.w[j] * fv : fv;
        }
      } else {
        const int fyi = side == 2 ? iy : iyT;
#pragma unroll
        for (int j = 0; j < n; ++j)
          acc += tb.w[j] * P.b.fy[v * nYf + ((size_t)fyi * m.nx + ix) * n + j];
      }
      fI[el * NSIDE * M + t] = acc;
    }
    elem_reduce<NP, M>(fRed, epb, el, k, OpSum());
    // conservative FP64 mean update of eq. (upmean): one thread per (element,
    // variable), the block's elements side by side in its first threads
    for (int t = tid; t < epb * M; t += T) {
      const int e2 = t / M, v = t - e2 * M;
      const int eg0 = blk * epr + e2;
      const int eg = (e2 < epr && eg0 < m.ne) ? eg0 : m.ne - 1;
      const real* I = fI + e2 * NSIDE * M;
      double mv = P.b.umean[(size_t)v * m.ne + eg] + dtd * P.b.smean[(size_t)v * m.ne + eg] -
                  dtd * m.invdx * (double(I[1 * M + v]) - double(I[0 * M + v]));
      if (DIM == 2) mv -= dtd * m.invdy * (double(I[3 * M + v]) - double(I[2 * M + v]));
      sEl[e2 * 16 + 4 + v] = mv;
      sElr[e2 * ES + ER + 1 + v] = real(mv);  // copy in the kernel's type
    }
#pragma unroll
    for (int v = 0; v < M; ++v) m32[v] = fRed[(v * epb + el) * NP];
    __syncthreads();
#pragma unroll
    for (int v = 0; v < M; ++v) ubar[v] = sEl[el * 16 + 4 + v];
  } else {
#pragma unroll
    for (int v = 0; v < M; ++v) RED(v) = double(W) * double(val[v]);
    elem_reduce<NP, M>(sRed, epb, el, k, OpSum());
#pragma unroll
    for (int v = 0; v < M; ++v) ubar[v] = RED0(v);
    for (int v = k; v < M; v += NP) sEl[el * 16 + 4 + v] = RED0(v);  // for the CFL rate
  }
  // node value in the kernel's type (FP64 mode the update itself; FP32_BULK the
  // FP64 mean plus the re-centred FP32 fluctuation), stored for the face traces of
  // the scaling limiter; the barrier after the limiter scalars covers it (sU is
  // free here: the face-flux integrals it held are consumed)
  real fl[M];
  real ur[M];
  real ubr[M];  // mean in the kernel's type
#pragma unroll
  for (int v = 0; v < M; ++v) {
    if constexpr (MIXED) ubr[v] = sElr[el * ES + ER + 1 + v];
    else ubr[v] = real(ubar[v]);
    if constexpr (MIXED) {
      fl[v] = val[v] - m32[v];
      ur[v] = ubr[v] + fl[v];
    } else {
      ur[v] = val[v];
    }
  }
  real* sUr = reinterpret_cast<real*>(sU);
#pragma unroll
  for (int v = 0; v < M; ++v) sUr[v * stride + el * NP + k] = ur[v];
  // per-element limiter scalars: sEl[el*16 + 0..3] = mean_ok, eps1, eps2, P2(u_bar),
  // for the block's elements side by side in its first epb threads (one warp)
  // from the means in shared memory.  FP32_BULK: when the FP32 copy of the mean
  // is clearly admissible the FP64 values are known without FP64 work (eps =
  // 1e-12); otherwise FP64.
  if (threadIdx.x < epb) {
    const int e2 = threadIdx.x;
    double ub2[M];
#pragma unroll
    for (int v = 0; v < M; ++v) ub2[v] = MIXED ? sEl[e2 * 16 + 4 + v] : sRed[(v * epb + e2) * NP];
    bool done = false;
    if constexpr (MIXED) {
      if (EQ::K > 0) {
        real ub[M];
#pragma unroll
        for (int v = 0; v < M; ++v) ub[v] = sElr[e2 * ES + ER + 1 + v];
        const real scale = EQ::M == 6 ? fabs(ub[3]) + fabs(ub[5]) : fabs(ub[M - 1]);
        const real P2f = EQ::constraint(ub, 1, P.ph);
        if (ub[0] > real(1e-9) && P2f > real(1e-5) * scale + real(1e-9)) {
          sEl[e2 * 16 + 0] = 1.0;
          sEl[e2 * 16 + 1] = 1e-12;
          sEl[e2 * 16 + 2] = 1e-12;
          sEl[e2 * 16 + 3] = double(P2f);
          done = true;
        }
      }
    }
    if (!done) {
      const double P2 = EQ::K > 0 ? EQ::constraint(ub2, 1, P.phd) : 0.0;
      sEl[e2 * 16 + 0] = admissible<EQ>(ub2, P.phd) ? 1.0 : 0.0;
      sEl[e2 * 16 + 1] = EQ::K > 0 ? fmin(1e-12, ub2[0]) : 0.0;
      sEl[e2 * 16 + 2] = EQ::K > 0 ? fmin(1e-12, P2) : 0.0;
      sEl[e2 * 16 + 3] = P2;
    }
    if constexpr (MIXED) {  // FP32 copies of P2(u_bar) and mean_ok for the node threads
      sElr[e2 * ES + ER + 7] = real(sEl[e2 * 16 + 3]);
      sElr[e2 * ES + ER + 8] = sEl[e2 * 16 + 0] != 0.0 ? real(1) : real(0);
    }
  }
  __syncthreads();

  // ---- positivity scaling limiter (FP64 theta) ----------------------------
  int bad = 0;
  const bool mean_ok = MIXED ? sElr[el * ES + ER + 8] != real(0) : sEl[el * 16 + 0] != 0.0;
  if (EQ::K > 0 && !mean_ok) bad |= kStInadmissible;
  const bool do_scale = (m.limiter & kLimScaling) && EQ::K > 0;
  const bool traces = (m.limiter & kLimTraces) != 0;
  if (do_scale) {
    const double eps1 = sEl[el * 16 + 1], eps2 = sEl[el * 16 + 2];
    const real P2r = MIXED ? sElr[el * ES + ER + 7] : real(sEl[el * 16 + 3]);
    // points this thread checks: its node and its face-trace slots
    real pr[1 + SPT][M];
    int npt = 1;
#pragma unroll
    for (int v = 0; v < M; ++v) pr[0][v] = ur[v];
    if (traces) {
#pragma unroll
      for (int mm = 0; mm < SPT; ++mm) {
        const int sl = k + mm * NP;
        if (sl < NSLOT) {
          const int side = sl / NFN, j = sl - side * NFN;
#pragma unroll
          for (int v = 0; v < M; ++v) {
            real acc = real(0);
#pragma unroll
            for (int r = 0; r < n; ++r) {
              const real l = (side & 1) ? tb.l1[r] : tb.l0[r];
              acc += l * sUr[v * stride + el * NP + (side < 2 ? r + n * j : j + n * r)];
            }
            pr[npt][v] = acc;
          }
          ++npt;
        }
      }
    }
    // does any point of the block need limiting?  FP64 mode: exactly the
    // oracle's test; FP32_BULK: an FP32 prescreen with a margin, the FP64
    // solve below decides
    int need = 0;
    for (int t = 0; t < npt; ++t) {
      if constexpr (MIXED) {
        const real scale = EQ::M == 6 ? fabs(pr[t][3]) + fabs(pr[t][5]) : fabs(pr[t][M - 1]);
        const real thr = fmax(fmax(real(1e-3) * P2r, real(1e-5) * scale), real(1e-11));
        if (!(pr[t][0] > real(1e-3) * ubr[0] && EQ::constraint(pr[t], 1, P.ph) > thr)) need = 1;
      } else {
        if (!(pr[t][0] >= eps1 && EQ::constraint(pr[t], 1, P.phd) >= eps2)) need = 1;
      }
    }
    // Only real elements vote (a ghost slot of a block whose size is not a
    // multiple of the element size holds partial data), and only an element
    // with a failing point takes the FP64 result below: the others keep their
    // values bit for bit, whichever elements share their block.
    if (__syncthreads_or(valid && need)) {
      // FP64 path (oracle's limiter): points in FP64
      double pts[1 + SPT][M];
      int np2 = 1;
      __syncthreads();
      RED(0) = need ? 0.0 : 1.0;
      elem_reduce<NP, 1>(sRed, epb, el, k, OpMin());
      const bool elem_need = RED0(0) == 0.0;
      __syncthreads();
#pragma unroll
      for (int v = 0; v < M; ++v) {
        if constexpr (MIXED) pts[0][v] = ubar[v] + double(fl[v]);
        else pts[0][v] = double(ur[v]);
      }
#pragma unroll
      for (int v = 0; v < M; ++v) ATU(v, k) = pts[0][v];
      __syncthreads();
      if (traces) {
#pragma unroll
        for (int mm = 0; mm < SPT; ++mm) {
          const int sl = k + mm * NP;
          if (sl < NSLOT) {
            const int side = sl / NFN, j = sl - side * NFN;
#pragma unroll
            for (int v = 0; v < M; ++v) {
              double acc = 0.0;
#pragma unroll
              for (int r = 0; r < n; ++r) {
                const double l = (side & 1) ? td.l1[r] : td.l0[r];
                acc += l * ATU(v, side < 2 ? r + n * j : j + n * r);
              }
              pts[np2][v] = acc;
            }
            ++np2;
          }
        }
      }
      double rmin = pts[0][0];
      for (int t = 1; t < np2; ++t) rmin = fmin(rmin, pts[t][0]);
      RED(0) = rmin;
      elem_reduce<NP, 1>(sRed, epb, el, k, OpMin());
      rmin = RED0(0);
      __syncthreads();
      if (mean_ok && rmin < eps1) {
        const double th1 = (ubar[0] - eps1) / (ubar[0] - rmin);
        for (int t = 0; t < np2; ++t) pts[t][0] = ubar[0] + th1 * (pts[t][0] - ubar[0]);
      }
      double tmin = 1.0;
      if (mean_ok)
        for (int t = 0; t < np2; ++t) {
          if (EQ::constraint(pts[t], 1, P.phd) >= eps2) continue;
          double lo = 0.0, hi = 1.0, tmp[M];
          for (int it = 0; it < 50; ++it) {
            const double mid = 0.5 * (lo + hi);
#pragma unroll
            for (int v = 0; v < M; ++v) tmp[v] = ubar[v] + mid * (pts[t][v] - ubar[v]);
            if (EQ::constraint(tmp, 1, P.phd) >= eps2) lo = mid;
            else hi = mid;
          }
          tmin = fmin(tmin, lo);
        }
      RED(0) = tmin;
      elem_reduce<NP, 1>(sRed, epb, el, k, OpMin());
      const double th2 = RED0(0);
      __syncthreads();
      if (th2 < 1.0)
        for (int t = 0; t < np2; ++t)
#pragma unroll
          for (int v = 0; v < M; ++v) pts[t][v] = ubar[v] + th2 * (pts[t][v] - ubar[v]);
      // status tests only the mean (above): the limited points are admissible
      // in exact arithmetic, and a tiny constraint value at a face trace is
      // below the rounding of its interpolation
      if (elem_need) {
#pragma unroll
        for (int v = 0; v < M; ++v) {
          if constexpr (MIXED) fl[v] = real(pts[0][v] - ubar[v]);
          ur[v] = real(pts[0][v]);
        }
      }
    }
  }
#pragma unroll
  for (int v = 0; v < M; ++v)
    if (!isfinite(ur[v])) bad |= kStNonFinite;
  if (valid && bad) {
    atomicOr(&P.b.ctl->status, bad);
    atomicMin(&P.b.ctl->bad_elem, e);
  }
  if (valid) {
#pragma unroll
    for (int v = 0; v < M; ++v) {
      const size_t gi = ((size_t)v * m.ne + e) * NP + k;
      if constexpr (MIXED) P.b.u[gi] = fl[v];
      else P.b.u[gi] = ur[v];
    }
    if constexpr (MIXED) {
      for (int v = k; v < M; v += NP) {
        P.b.umean[(size_t)v * m.ne + e] = ubar[v];
        P.b.umean_f[(size_t)v * m.ne + e] = float(ubar[v]);
      }
    }
    // cr_step_get: the new state in FP64 straight into the caller's host
    // memory (the transfer overlaps the rest of the kernel); FP32 bulk as
    // mean + fluctuation, the sum the state read-back forms
    double* const out = deferred ? P.b.ctl->out : nullptr;
    if (out) {
#pragma unroll
      for (int v = 0; v < M; ++v) {
        const size_t gi = ((size_t)v * m.ne + e) * NP + k;
        if constexpr (MIXED) out[gi] = ubar[v] + double(fl[v]);
        else out[gi] = double(ur[v]);
      }
    }
  }

  // ---- indicator of the new state and the CFL rate -------------------------
  if ((m.limiter & kLimBlend) && (m.alpha_mode == 0 || m.alpha_mode == 2)) {
    if constexpr (MIXED) {
      real* rE = reinterpret_cast<real*>(sU);
      real* rT = rE + stride;
      real* rR = rT + stride;
      __syncthreads();
      rE[el * NP + k] = EQ::indicator_var(ur, P.ph);
      __syncthreads();
      const real al = indicator_alpha<DIM, N, real>(m, tb, rE, rT, rR, epb, el, k, P.b.mlp_flag,
                                                    P.b.mlp_w, sMlp, nullptr, -1);
      if (valid && k == 0) {
        P.b.alpha_raw[e] = double(al);
        P.b.alpha_raw_f[e] = al;
      }
    } else {
      double* dE = sU;
      double* dT = sU + stride;
      __syncthreads();
      dE[el * NP + k] = EQ::indicator_var(ur, P.phd);
      __syncthreads();
      const double al = indicator_alpha<DIM, N, double>(m, td, dE, dT, sRed, epb, el, k,
                                                        P.b.mlp_flag, P.b.mlp_w, sMlp, nullptr, -1);
      if (valid && k == 0) P.b.alpha_raw[e] = al;
    }
  }
  __syncthreads();
  if constexpr (MIXED) {
    rate_and_finish<DIM, NP, EQ, float>(m, P.ph, sElr + ER + 1, ES, reinterpret_cast<float*>(sRed),
                                        epb, epr, blk * epr, P.b.ctl, 1, dtd, last_step, nblk, tb.xi,
                                        deferred);
  } else {
    rate_and_finish<DIM, NP, EQ, double>(m, P.phd, sEl + 4, 16, sRed, epb, epr, blk * epr, P.b.ctl, 1,
                                         dtd, last_step, nblk, td.xi, deferred);
  }
#undef ATU
#undef RED
#undef RED0
}

template <int DIM, int N, class EQ, typename real, bool MIXED>
__global__ void __launch_bounds__(256, MinBlocks<MIXED>::update) k_update(const __grid_constant__ KParams<real> P) {
  update_body<DIM, N, EQ, real, MIXED, UpdateShape<DIM == 2 ? (N + 1) * (N + 1) : N + 1, MIXED>::T>(
      P, P.tb, P.td, blockIdx.x, gridDim.x, true);  // k_finish_step ends the step
}

// ===========================================================================
// After cr_set_state: validate the input, compute the indicator of the state
// and the CFL rate of eq. (time.step.2d) (no time advance).
template <int DIM, int N, class EQ, typename real, bool MIXED>
__global__ void k_prologue(const __grid_constant__ KParams<real> P) {
  constexpr int n = N + 1;
  constexpr int NP = DIM == 2 ? n * n : n;
  constexpr int M = EQ::M;
  constexpr int RW = 2 * M > 4 ? 2 * M : 4;
  constexpr int MU = M > 2 ? M : 2;
  const Mesh& m = P.m;
  const int epb = (blockDim.x + NP - 1) / NP;  // element slots in shared memory
  const int epr = blockDim.x / NP;             // whole elements of the block
  const int tid = threadIdx.x;
  const int el = tid / NP, k = tid - el * NP;
  const int e = blockIdx.x * epr + el;
  const bool valid = el < epr && e < m.ne;
  const int ee = valid ? e : m.ne - 1;
  const int stride = epb * NP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sU = reinterpret_cast<double*>(smem_raw);
  double* sRed = sU + MU * stride;
  double* sEl = sRed + RW * stride;
  float* sMlp = reinterpret_cast<float*>(sEl + 16 * epb);
  const int p = DIM == 2 ? k % n : k, q = DIM == 2 ? k / n : 0;
  const double W = DIM == 2 ? P.td.w[p] * P.td.w[q] : P.td.w[p];
  double u[M];
  int bad = 0;
#pragma unroll
  for (int v = 0; v < M; ++v) {
    const size_t gi = ((size_t)v * m.ne + ee) * NP + k;
    if constexpr (!MIXED) {
      if (P.b.u_src) {  // the state straight from pinned host memory: load once, keep a copy
        u[v] = P.b.u_src[gi];
        if (valid) P.b.u[gi] = real(u[v]);
      } else {
        u[v] = double(P.b.u[gi]);
      }
    } else {
      u[v] = double(P.b.u[gi]) + P.b.umean[(size_t)v * m.ne + ee];
    }
    if (!isfinite(u[v])) bad = kStInvalidInput;
    sRed[(v * epb + el) * NP + k] = W * u[v];
  }
  if (!admissible<EQ>(u, P.phd)) bad = kStInvalidInput;
  if (valid && bad) {
    atomicOr(&P.b.ctl->status, bad);
    atomicMin(&P.b.ctl->bad_elem, e);
  }
  elem_reduce<NP, M>(sRed, epb, el, k, OpSum());
  double ubar[M];
#pragma unroll
  for (int v = 0; v < M; ++v) ubar[v] = sRed[(v * epb + el) * NP];
  for (int v = k; v < M; v += NP) sEl[el * 16 + 4 + v] = ubar[v];  // for the CFL rate
  __syncthreads();
  if (((m.limiter & kLimBlend) && (m.alpha_mode == 0 || m.alpha_mode == 2)) || P.b.feat) {
    sU[el * NP + k] = EQ::indicator_var(u, P.phd);
    __syncthreads();
    const double al = indicator_alpha<DIM, N, double>(m, P.td, sU, sU + stride, sRed, epb, el, k,
                                                      P.b.mlp_flag, P.b.mlp_w, sMlp, P.b.feat,
                                                      valid ? e : -1);
    if (valid && k == 0) {
      P.b.alpha_raw[e] = al;
      if constexpr (MIXED) P.b.alpha_raw_f[e] = float(al);
    }
  }
  __syncthreads();
  rate_and_finish<DIM, NP, EQ, double>(m, P.phd, sEl + 4, 16, sRed, epb, epr, blockIdx.x * epr, P.b.ctl,
                                       0, 0.0, 0, gridDim.x, P.td.xi);
}

// FP32_BULK state conversion: FP64 nodal values <-> FP64 mean + FP32 fluctuation.
template <int DIM, int N, int M>
__global__ void k_split_state(const double* __restrict__ in, float* __restrict__ fl,
                              double* __restrict__ mean, float* __restrict__ mean_f, int ne,
                              Tab<double> td) {
  constexpr int n = N + 1;
  constexpr int NP = DIM == 2 ? n * n : n;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // one thread per (v, e)
  if (idx >= M * ne) return;
  const double* x = in + (size_t)idx * NP;
  double mu = 0.0;
  for (int kk = 0; kk < NP; ++kk) {
    const int pp = DIM == 2 ? kk % n : kk, qq = DIM == 2 ? kk / n : 0;
    mu += (DIM == 2 ? td.w[pp] * td.w[qq] : td.w[pp]) * x[kk];
  }
  mean[idx] = mu;
  mean_f[idx] = float(mu);
  for (int kk = 0; kk < NP; ++kk) fl[(size_t)idx * NP + kk] = float(x[kk] - mu);
}

// Element means sum_k W_k u_k of an FP64 state [M][Ne][Np] -> [M][Ne].
template <int DIM, int N, int M>
__global__ void k_element_means(const double* __restrict__ u, double* __restrict__ mean, int ne,
                                Tab<double> td) {
  constexpr int n = N + 1;
  constexpr int NP = DIM == 2 ? n * n : n;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // one thread per (v, e)
  if (idx >= M * ne) return;
  const double* x = u + (size_t)idx * NP;
  double mu = 0.0;
  for (int kk = 0; kk < NP; ++kk) {
    const int pp = DIM == 2 ? kk % n : kk, qq = DIM == 2 ? kk / n : 0;
    mu += (DIM == 2 ? td.w[pp] * td.w[qq] : td.w[pp]) * x[kk];
  }
  mean[idx] = mu;
}

template <int NP>
__global__ void k_join_state(const float* __restrict__ fl, const double* __restrict__ mean,
                             double* __restrict__ out, int nvals) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // one thread per value
  if (idx >= nvals) return;
  out[idx] = mean[idx / NP] + double(fl[idx]);
}

}  // namespace crk
