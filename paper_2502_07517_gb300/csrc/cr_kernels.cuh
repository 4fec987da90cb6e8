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

template <typename real>
__device__ __forceinline__ real minmod3(real a, real b, real c) {
  if (a > real(0) && b > real(0) && c > real(0)) return fmin(a, fmin(b, c));
  if (a < real(0) && b < real(0) && c < real(0)) return fmax(a, fmax(b, c));
  return real(0);
}

template <class EQ, typename real>
__device__ __forceinline__ bool admissible(const real* u, const Mesh& m) {
  bool ok = true;
#pragma unroll
  for (int k = 0; k < EQ::K; ++k) ok = ok && (EQ::constraint(u, k, m) > real(0));
  return ok;
}

// Rusanov flux, Sec. 2 eqs. (num.flux.fr), (rusanov.wave.speed).
template <class EQ, typename real>
__device__ __forceinline__ void rusanov(const real* uL, const real* uR, int dir, real* out,
                                        const Mesh& m) {
  real fL[EQ::M], fR[EQ::M];
  EQ::flux(uL, dir, fL, m);
  EQ::flux(uR, dir, fR, m);
  real lam = fmax(EQ::speed(uL, dir, m), EQ::speed(uR, dir, m));
#pragma unroll
  for (int v = 0; v < EQ::M; ++v)
    out[v] = real(0.5) * (fL[v] + fR[v]) - real(0.5) * lam * (uR[v] - uL[v]);
}

// Load variable v of node k of element e from the state (mean + fluctuation
// in FP32_BULK mode).
template <typename real, bool MIXED>
__device__ __forceinline__ real load_state(const Bufs<real>& b, int ne, int NP, int v, int e,
                                           int k) {
  const real x = b.u[((size_t)v * ne + e) * NP + k];
  if constexpr (MIXED) return real(b.umean[(size_t)v * ne + e] + double(x));
  return x;
}

// slot buffer index: field f (0 sigma, 1.. U, 1+M.. EA, 1+2M.. u*, 1+3M.. base)
__device__ __forceinline__ size_t slot_index(int f, int side, int e, int j, int nside, int ne,
                                             int nfn) {
  return (((size_t)f * nside + side) * ne + e) * nfn + j;
}

// ===========================================================================
template <int DIM, int N, class EQ, typename real, bool MIXED>
__global__ void k_local(const KParams<real> P) {
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
  const Tab<real>& tb = P.tb;
  const int epb = blockDim.x / NP;
  const int tid = threadIdx.x;
  const int el = tid / NP, k = tid - el * NP;
  const int p = DIM == 2 ? k % n : k, q = DIM == 2 ? k / n : 0;
  const int e = blockIdx.x * epb + el;
  const bool valid = e < m.ne;
  const int ee = valid ? e : m.ne - 1;
  const int ix = ee % m.nx, iy = ee / m.nx;

  bool last;
  const double dtd = step_dt(P.b.ctl, &last);
  if (blockIdx.x == 0 && tid == 0) {
    P.b.ctl->dt_step = dtd > 0.0 ? dtd : 0.0;
    P.b.ctl->last_step = last ? 1 : 0;
  }
  if (!(dtd > 0.0)) return;
  const real dt = real(dtd);

  extern __shared__ __align__(16) unsigned char smem_raw[];
  real* sh = reinterpret_cast<real*>(smem_raw);
  const int stride = epb * NP;
  const int arr = M * stride;
  real* s0 = sh;
  real* sA = sh + arr;
  real* sB = sA + arr;
  real* sC = sB + arr;
  real* sD = sC + arr;
#define AT(base, v, node) base[(v) * stride + el * NP + (node)]

  real un[M];
#pragma unroll
  for (int v = 0; v < M; ++v) {
    un[v] = load_state<real, MIXED>(P.b, m.ne, NP, v, ee, k);
    AT(s0, v, k) = un[v];
  }

  // blending coefficient alpha_e, smoothed with the face neighbours
  double alpha = 0.0;
  if (m.alpha_mode == 1) {
    alpha = m.alpha_fixed;
  } else if (m.limiter & kLimBlend) {
    alpha = P.b.alpha_raw[ee];
#pragma unroll
    for (int f = 0; f < NSIDE; ++f) {
      const int nb = neighbour(m, ee, f);
      if (nb >= 0) alpha = fmax(alpha, 0.5 * P.b.alpha_raw[nb]);
    }
  }
  if (valid && k == 0) P.b.alpha[e] = alpha;
  const bool blend = (m.limiter & kLimBlend) || m.alpha_mode == 1;
  const bool need_lo = blend || (m.limiter & kLimFlux);
  const real a = blend ? real(alpha) : real(0);

  // source: grad W at this node (time independent)
  const bool has_src = (EQ::M == 6) && m.source == 1;
  real dWx = real(0), dWy = real(0);
  if (has_src) {
    double x = m.x0 + (ix + double(tb.xi[p])) * m.dx;
    double y = DIM == 2 ? m.y0 + (iy + double(tb.xi[q])) * m.dy : 0.0;
    double gx, gy;
    source_grad<DIM>(m, x, y, &gx, &gy);
    dWx = real(gx);
    dWy = real(gy);
  }

  // ---------------- local cRK stages -----------------------------------
  real Lst[S > 1 ? S - 1 : 1][M];
  real Fa[M], Ga[M], Ua[M], Sa[M];
  real ea[SPT][M];
#pragma unroll
  for (int v = 0; v < M; ++v) {
    Fa[v] = Ga[v] = Ua[v] = Sa[v] = real(0);
#pragma unroll
    for (int mm = 0; mm < SPT; ++mm) ea[mm][v] = real(0);
  }
  const real invdx = real(m.invdx), invdy = real(m.invdy);

#pragma unroll
  for (int i = 0; i < S; ++i) {
    real ui[M];
#pragma unroll
    for (int v = 0; v < M; ++v) {
      real acc = un[v];
#pragma unroll
      for (int j = 0; j < i; ++j)
        if (TB::a(i, j) != 0.0) acc -= (dt * real(TB::a(i, j))) * Lst[j][v];
      ui[v] = acc;
    }
    real f[M], g[M], s[M];
    EQ::flux(ui, 0, f, m);
    if (DIM == 2) EQ::flux(ui, 1, g, m);
    if (has_src) source_eval<EQ>(ui, dWx, dWy, s);
    else {
#pragma unroll
      for (int v = 0; v < M; ++v) s[v] = real(0);
    }
    if (TB::b(i) != 0.0) {
      const real bi = real(TB::b(i));
#pragma unroll
      for (int v = 0; v < M; ++v) {
        Fa[v] += bi * f[v];
        if (DIM == 2) Ga[v] += bi * g[v];
        Ua[v] += bi * ui[v];
        Sa[v] += bi * s[v];
      }
    }
#pragma unroll
    for (int v = 0; v < M; ++v) {
      AT(sA, v, k) = ui[v];
      AT(sB, v, k) = f[v];
      if (DIM == 2) AT(sC, v, k) = g[v];
    }
    __syncthreads();
    if (i < S - 1) {
#pragma unroll
      for (int v = 0; v < M; ++v) {
        real hx = real(0), hy = real(0);
#pragma unroll
        for (int r = 0; r < n; ++r) hx += tb.D[p * n + r] * AT(sB, v, r + n * q);
        if (DIM == 2) {
#pragma unroll
          for (int r = 0; r < n; ++r) hy += tb.D[q * n + r] * AT(sC, v, p + n * r);
        }
        Lst[i < S - 1 ? i : 0][v] = invdx * hx + (DIM == 2 ? invdy * hy : real(0)) - s[v];
      }
    }
    if (TB::b(i) != 0.0) {
      const real bi = real(TB::b(i));
#pragma unroll
      for (int mm = 0; mm < SPT; ++mm) {
        const int sl = k + mm * NP;
        if (sl < NSLOT) {
          const int side = sl / NFN, j = sl - side * NFN;
          real ut[M], fn[M];
#pragma unroll
          for (int v = 0; v < M; ++v) {
            real acc = real(0);
#pragma unroll
            for (int r = 0; r < n; ++r) {
              const real l = (side & 1) ? tb.l1[r] : tb.l0[r];
              acc += l * AT(sA, v, side < 2 ? r + n * j : j + n * r);
            }
            ut[v] = acc;
          }
          EQ::flux(ut, side >> 1, fn, m);
#pragma unroll
          for (int v = 0; v < M; ++v) ea[mm][v] += bi * fn[v];
        }
      }
    }
    __syncthreads();
  }

  // ---------------- time averages: high-order volume part, face data ----
#pragma unroll
  for (int v = 0; v < M; ++v) {
    AT(sA, v, k) = Ua[v];
    AT(sB, v, k) = Fa[v];
    if (DIM == 2) AT(sC, v, k) = Ga[v];
  }
  __syncthreads();
  real HO[M];
#pragma unroll
  for (int v = 0; v < M; ++v) {
    real hx = real(0), hy = real(0);
#pragma unroll
    for (int r = 0; r < n; ++r) hx += tb.Dt[p * n + r] * AT(sB, v, r + n * q);
    if (DIM == 2) {
#pragma unroll
      for (int r = 0; r < n; ++r) hy += tb.Dt[q * n + r] * AT(sC, v, p + n * r);
    }
    HO[v] = invdx * hx + (DIM == 2 ? invdy * hy : real(0));
  }
#pragma unroll
  for (int mm = 0; mm < SPT; ++mm) {
    const int sl = k + mm * NP;
    if (valid && sl < NSLOT) {
      const int side = sl / NFN, j = sl - side * NFN;
      real Ut[M], ut[M];
#pragma unroll
      for (int v = 0; v < M; ++v) {
        real a1 = real(0), a2 = real(0);
#pragma unroll
        for (int r = 0; r < n; ++r) {
          const real l = (side & 1) ? tb.l1[r] : tb.l0[r];
          const int node = side < 2 ? r + n * j : j + n * r;
          a1 += l * AT(sA, v, node);
          a2 += l * AT(s0, v, node);
        }
        Ut[v] = a1;
        ut[v] = a2;
      }
      real* sl_out = P.b.slot;
      sl_out[slot_index(0, side, e, j, NSIDE, m.ne, NFN)] = EQ::speed(ut, side >> 1, m);
#pragma unroll
      for (int v = 0; v < M; ++v) {
        sl_out[slot_index(1 + v, side, e, j, NSIDE, m.ne, NFN)] = Ut[v];
        sl_out[slot_index(1 + M + v, side, e, j, NSIDE, m.ne, NFN)] = ea[mm][v];
      }
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
      const real beta = real(2.0 - alpha);
      real um[M], up[M], sx[M], sy[M];
      // x-line neighbours (the neighbour element's node across a face; own node at outflow)
      const int nbL = p == 0 ? neighbour(m, ee, 0) : -1;
      const int nbR = p == N ? neighbour(m, ee, 1) : -1;
#pragma unroll
      for (int v = 0; v < M; ++v) {
        um[v] = p > 0 ? AT(s0, v, k - 1)
                      : (nbL >= 0 ? load_state<real, MIXED>(P.b, m.ne, NP, v, nbL, N + n * q) : un[v]);
        up[v] = p < N ? AT(s0, v, k + 1)
                      : (nbR >= 0 ? load_state<real, MIXED>(P.b, m.ne, NP, v, nbR, n * q) : un[v]);
        sx[v] = minmod3(beta * (un[v] - um[v]) * tb.ihm[p], (up[v] - um[v]) * tb.ihc[p],
                        beta * (up[v] - un[v]) * tb.ihp[p]);
        sy[v] = real(0);
      }
      if (DIM == 2) {
        const int nbB = q == 0 ? neighbour(m, ee, 2) : -1;
        const int nbT = q == N ? neighbour(m, ee, 3) : -1;
#pragma unroll
        for (int v = 0; v < M; ++v) {
          um[v] = q > 0 ? AT(s0, v, k - n)
                        : (nbB >= 0 ? load_state<real, MIXED>(P.b, m.ne, NP, v, nbB, p + n * N) : un[v]);
          up[v] = q < N ? AT(s0, v, k + n)
                        : (nbT >= 0 ? load_state<real, MIXED>(P.b, m.ne, NP, v, nbT, p) : un[v]);
          sy[v] = minmod3(beta * (un[v] - um[v]) * tb.ihm[q], (up[v] - um[v]) * tb.ihc[q],
                          beta * (up[v] - un[v]) * tb.ihp[q]);
        }
      }
      real fxm[M], fxp[M], fym[M], fyp[M], Fm[M], Fp[M], Gm[M], Gp[M];
#pragma unroll
      for (int v = 0; v < M; ++v) {
        fxm[v] = un[v] + sx[v] * tb.dm[p];
        fxp[v] = un[v] + sx[v] * tb.dp[p];
        fym[v] = un[v] + sy[v] * tb.dm[q];
        fyp[v] = un[v] + sy[v] * tb.dp[q];
      }
      EQ::flux(fxm, 0, Fm, m);
      EQ::flux(fxp, 0, Fp, m);
      if (DIM == 2) {
        EQ::flux(fym, 1, Gm, m);
        EQ::flux(fyp, 1, Gp, m);
      }
      real ex[M], exm[M], exp_[M], eym[M], eyp[M];
#pragma unroll
      for (int v = 0; v < M; ++v) {
        ex[v] = real(0.5) * dt * (Fp[v] - Fm[v]) * tb.invw[p] * invdx;
        if (DIM == 2) ex[v] += real(0.5) * dt * (Gp[v] - Gm[v]) * tb.invw[q] * invdy;
        exm[v] = fxm[v] - ex[v];
        exp_[v] = fxp[v] - ex[v];
        eym[v] = fym[v] - ex[v];
        eyp[v] = fyp[v] - ex[v];
      }
      bool ok = admissible<EQ>(fxm, m) && admissible<EQ>(fxp, m) && admissible<EQ>(exm, m) &&
                admissible<EQ>(exp_, m);
      if (DIM == 2)
        ok = ok && admissible<EQ>(fym, m) && admissible<EQ>(fyp, m) && admissible<EQ>(eym, m) &&
             admissible<EQ>(eyp, m);
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
#pragma unroll
    for (int v = 0; v < M; ++v) {
      AT(sA, v, k) = xm[v];
      AT(sB, v, k) = xp[v];
      if (DIM == 2) {
        AT(sC, v, k) = ym[v];
        AT(sD, v, k) = yp[v];
      }
    }
    __syncthreads();
    // subcell fluxes: thread (p,q) owns the subface to its right (x) and top (y);
    // its own x+ (y+) state is read only by itself, so it is overwritten in place
    if (p < N) {
      real uL[M], uR[M], fr[M];
#pragma unroll
      for (int v = 0; v < M; ++v) {
        uL[v] = AT(sB, v, k);
        uR[v] = AT(sA, v, k + 1);
      }
      rusanov<EQ>(uL, uR, 0, fr, m);
#pragma unroll
      for (int v = 0; v < M; ++v) AT(sB, v, k) = fr[v];
    }
    if (DIM == 2 && q < N) {
      real uL[M], uR[M], fr[M];
#pragma unroll
      for (int v = 0; v < M; ++v) {
        uL[v] = AT(sD, v, k);
        uR[v] = AT(sC, v, k + n);
      }
      rusanov<EQ>(uL, uR, 1, fr, m);
#pragma unroll
      for (int v = 0; v < M; ++v) AT(sD, v, k) = fr[v];
    }
    __syncthreads();
    // low-order residual of the interior subfaces (eq. (low.order.update))
#pragma unroll
    for (int v = 0; v < M; ++v) {
      real rx = (p < N ? AT(sB, v, k) : real(0)) - (p > 0 ? AT(sB, v, k - 1) : real(0));
      LO[v] = rx * tb.invw[p] * invdx;
      if (DIM == 2) {
        real ry = (q < N ? AT(sD, v, k) : real(0)) - (q > 0 ? AT(sD, v, k - n) : real(0));
        LO[v] += ry * tb.invw[q] * invdy;
      }
    }
    // face-node data for the face kernel: evolved boundary state u* and the
    // candidate base of the flux limiter, u_b -+ c f_adj
    const double kappa = DIM == 2 ? 0.5 : 1.0;
#pragma unroll
    for (int mm = 0; mm < SPT; ++mm) {
      const int sl = k + mm * NP;
      if (valid && sl < NSLOT) {
        const int side = sl / NFN, j = sl - side * NFN;
        int nb_node, adj_node;
        const real* ust;
        const real* adj;
        if (side == 0) { nb_node = n * j; adj_node = n * j; ust = sA; adj = sB; }
        else if (side == 1) { nb_node = N + n * j; adj_node = N - 1 + n * j; ust = sB; adj = sB; }
        else if (side == 2) { nb_node = j; adj_node = j; ust = sC; adj = sD; }
        else { nb_node = j + n * N; adj_node = j + n * (N - 1); ust = sD; adj = sD; }
        const double h = side < 2 ? m.dx : m.dy;
        const double c = dtd / (kappa * P.td.w[(side & 1) ? N : 0] * h);
        const double sgn = (side & 1) ? 1.0 : -1.0;
#pragma unroll
        for (int v = 0; v < M; ++v) {
          P.b.slot[slot_index(1 + 2 * M + v, side, e, j, NSIDE, m.ne, NFN)] =
              ust[v * stride + el * NP + nb_node];
          P.b.slot[slot_index(1 + 3 * M + v, side, e, j, NSIDE, m.ne, NFN)] =
              real(double(AT(s0, v, nb_node)) + sgn * c * double(adj[v * stride + el * NP + adj_node]));
        }
      }
    }
  }

  // ---------------- partial update --------------------------------------
  if (valid) {
#pragma unroll
    for (int v = 0; v < M; ++v) {
      const real val = un[v] - dt * ((real(1) - a) * HO[v] + a * LO[v]) + dt * Sa[v];
      P.b.P[((size_t)v * m.ne + e) * NP + k] = val;
    }
  }
  if constexpr (MIXED) {
    // FP64 source contribution to the element mean: sum_k W_k S_k
    __syncthreads();
#pragma unroll
    for (int v = 0; v < M; ++v) AT(sA, v, k) = Sa[v];
    __syncthreads();
    for (int v = k; valid && v < M; v += NP) {
      double acc = 0.0;
      for (int kk = 0; kk < NP; ++kk) {
        const int pp = DIM == 2 ? kk % n : kk, qq = DIM == 2 ? kk / n : 0;
        const double W = DIM == 2 ? P.td.w[pp] * P.td.w[qq] : P.td.w[pp];
        acc += W * double(sA[v * stride + el * NP + kk]);
      }
      P.b.smean[(size_t)v * m.ne + e] = acc;
    }
  }
#undef AT
}

// ===========================================================================
template <int DIM, int N, class EQ, typename real>
__global__ void k_face(const KParams<real> P) {
  constexpr int n = N + 1;
  constexpr int M = EQ::M;
  constexpr int NSIDE = DIM == 2 ? 4 : 2;
  constexpr int NFN = DIM == 2 ? n : 1;
  const Mesh& m = P.m;
  const double dtd = P.b.ctl->dt_step;
  if (!(dtd > 0.0)) return;
  const int nX = m.ny * m.nfx * NFN;
  const int nY = DIM == 2 ? m.nfy * m.nx * n : 0;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nX + nY) return;
  int dir, j, eL, eR;
  size_t out_idx, vstride;
  real* out;
  if (idx < nX) {
    dir = 0;
    j = idx % NFN;
    const int r = idx / NFN, i = r % m.nfx, iy = r / m.nfx;
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
  const real* sl = P.b.slot;
  auto fld = [&](int f, int side, int e) { return sl[slot_index(f, side, e, j, NSIDE, m.ne, NFN)]; };

  real FHO[M], fLO[M];
  double alpha_f;
  const bool blend = (m.limiter & kLimBlend) || m.alpha_mode == 1;
  const bool need_lo = blend || (m.limiter & kLimFlux);
  if (eL >= 0 && eR >= 0) {
    const real lam = fmax(fld(0, sL, eL), fld(0, sR, eR));
#pragma unroll
    for (int v = 0; v < M; ++v)
      FHO[v] = real(0.5) * (fld(1 + M + v, sL, eL) + fld(1 + M + v, sR, eR)) -
               real(0.5) * lam * (fld(1 + v, sR, eR) - fld(1 + v, sL, eL));
    if (need_lo) {
      real uL[M], uR[M];
#pragma unroll
      for (int v = 0; v < M; ++v) {
        uL[v] = fld(1 + 2 * M + v, sL, eL);
        uR[v] = fld(1 + 2 * M + v, sR, eR);
      }
      rusanov<EQ>(uL, uR, dir, fLO, m);
    }
    alpha_f = 0.5 * (P.b.alpha[eL] + P.b.alpha[eR]);
  } else {
    const int ei = eR >= 0 ? eR : eL;
    const int si = eR >= 0 ? sR : sL;
#pragma unroll
    for (int v = 0; v < M; ++v) FHO[v] = fld(1 + M + v, si, ei);
    if (need_lo) {
      real us[M];
#pragma unroll
      for (int v = 0; v < M; ++v) us[v] = fld(1 + 2 * M + v, si, ei);
      EQ::flux(us, dir, fLO, m);
    }
    alpha_f = P.b.alpha[ei];
  }
  double F[M];
#pragma unroll
  for (int v = 0; v < M; ++v)
    F[v] = blend ? (1.0 - alpha_f) * double(FHO[v]) + alpha_f * double(fLO[v]) : double(FHO[v]);
  double theta = 1.0;
  if ((m.limiter & kLimFlux) && EQ::K > 0) {
    const double kappa = DIM == 2 ? 0.5 : 1.0;
    const double h = dir == 0 ? m.dx : m.dy;
    const double cL = dtd / (kappa * P.td.w[N] * h), cR = dtd / (kappa * P.td.w[0] * h);
    double baseL[M], baseR[M], flo[M];
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
        PlowL = EQ::constraint(cand, kk, m);
        eps = fmin(eps, PlowL);
      }
      if (eR >= 0) {
#pragma unroll
        for (int v = 0; v < M; ++v) cand[v] = baseR[v] + cR * flo[v];
        PlowR = EQ::constraint(cand, kk, m);
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
        const double Pk = EQ::constraint(cand, kk, m);
        if (Pk < eps) tk = fmin(tk, (PlowL - eps) / (PlowL - Pk));
      }
      if (eR >= 0) {
#pragma unroll
        for (int v = 0; v < M; ++v) cand[v] = baseR[v] + cR * Ft[v];
        const double Pk = EQ::constraint(cand, kk, m);
        if (Pk < eps) tk = fmin(tk, (PlowR - eps) / (PlowR - Pk));
      }
      theta *= tk;
    }
#pragma unroll
    for (int v = 0; v < M; ++v) F[v] = theta * F[v] + (1.0 - theta) * flo[v];
  }
#pragma unroll
  for (int v = 0; v < M; ++v) out[v * vstride + out_idx] = real(F[v]);
}

// ===========================================================================
// Element-level helpers for k_update / k_prologue (one thread per node, EPB
// elements per block).  sRed: [EPB][NP] doubles.

// smoothness indicator of one element from eps at the nodes (in sE), returns alpha
// on thread k == 0; uses sT as scratch.  Modal energies: Legendre modes of eps,
// E = max(top-mode energy fraction, next-to-top fraction), logistic map.
template <int DIM, int N>
__device__ void indicator_alpha(const Mesh& m, const Tab<double>& td, double* sE, double* sT,
                                int el, int k, double* alpha_out) {
  constexpr int n = N + 1;
  constexpr int NP = DIM == 2 ? n * n : n;
  double* E = sE + el * NP;
  double* T = sT + el * NP;
  if (DIM == 2) {
    const int i = k % n, qq = k / n;
    double acc = 0.0;
#pragma unroll
    for (int pp = 0; pp < n; ++pp) acc += td.V[i * n + pp] * E[pp + n * qq];
    T[k] = acc;
    __syncthreads();
    const int jj = k / n;
    double mo = 0.0;
#pragma unroll
    for (int q2 = 0; q2 < n; ++q2) mo += td.V[jj * n + q2] * T[i + n * q2];
    __syncthreads();
    E[k] = mo * mo;
    __syncthreads();
  } else {
    double mo = 0.0;
#pragma unroll
    for (int pp = 0; pp < n; ++pp) mo += td.V[k * n + pp] * E[pp];
    __syncthreads();
    E[k] = mo * mo;
    __syncthreads();
  }
  if (k == 0) {
    double tot = 0.0, top = 0.0, low = 0.0, top1 = 0.0;
    for (int kk = 0; kk < NP; ++kk) {
      const int i = DIM == 2 ? kk % n : kk, j = DIM == 2 ? kk / n : 0;
      const int mx = i > j ? i : j;
      const double e2 = E[kk];
      tot += e2;
      if (mx == N) top += e2;
      if (mx <= N - 1) low += e2;
      if (mx == N - 1) top1 += e2;
    }
    const double r1 = tot > 0.0 ? top / tot : 0.0;
    const double r2 = (N >= 2 && low > 0.0) ? top1 / low : 0.0;
    const double Ev = fmax(r1, r2);
    double al = 1.0 / (1.0 + exp(-m.s_ind / m.T_ind * (Ev - m.T_ind)));
    if (al < 1e-3) al = 0.0;
    if (al > 1.0 - 1e-3) al = 1.0;
    *alpha_out = fmin(al, 1.0);
  }
}

// finish the step: block max of the CFL rate, last block publishes the rate,
// advances time when advance != 0, and resets the accumulators.
__device__ __forceinline__ void finish_block(TimeCtl* ctl, double block_rate, int advance,
                                             double dtd, int last_step) {
  if (threadIdx.x == 0) {
    atomicMax(&ctl->rate_acc, (unsigned long long)__double_as_longlong(block_rate));
    __threadfence();
    const unsigned prev = atomicAdd(&ctl->blocks_done, 1u);
    if (prev == gridDim.x - 1) {
      __threadfence();
      const unsigned long long bits = atomicExch(&ctl->rate_acc, 0ull);
      ctl->rate_last = __longlong_as_double((long long)bits);
      ctl->blocks_done = 0;
      if (advance) {
        ctl->t = last_step ? ctl->t_final : ctl->t + dtd;
        ctl->steps += 1;
      }
    }
  }
}

// ===========================================================================
template <int DIM, int N, class EQ, typename real, bool MIXED>
__global__ void k_update(const KParams<real> P) {
  constexpr int n = N + 1;
  constexpr int NP = DIM == 2 ? n * n : n;
  constexpr int M = EQ::M;
  constexpr int NSIDE = DIM == 2 ? 4 : 2;
  constexpr int NFN = DIM == 2 ? n : 1;
  constexpr int NSLOT = NSIDE * NFN;
  constexpr int SPT = (NSLOT + NP - 1) / NP;
  const Mesh& m = P.m;
  const Tab<double>& td = P.td;
  const double dtd = P.b.ctl->dt_step;
  const int last_step = P.b.ctl->last_step;
  if (!(dtd > 0.0)) return;
  const int epb = blockDim.x / NP;
  const int tid = threadIdx.x;
  const int el = tid / NP, k = tid - el * NP;
  const int p = DIM == 2 ? k % n : k, q = DIM == 2 ? k / n : 0;
  const int e = blockIdx.x * epb + el;
  const bool valid = e < m.ne;
  const int ee = valid ? e : m.ne - 1;
  const int ix = ee % m.nx, iy = ee / m.nx;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sU = reinterpret_cast<double*>(smem_raw);  // [M][epb][NP]
  double* sRed = sU + M * epb * NP;                  // [epb][NP]
  double* sT = sRed + epb * NP;                      // [epb][NP]
  double* sMean = sT + epb * NP;                     // [epb][M]
  double* sShift = sMean + epb * M;                  // [epb][M]
  double* sTh = sShift + epb * M;                    // [epb]
  const int stride = epb * NP;
#define ATU(v, node) sU[(v) * stride + el * NP + (node)]

  const double alpha = P.b.alpha[ee];
  const bool blend = (m.limiter & kLimBlend) || m.alpha_mode == 1;
  const real a = blend ? real(alpha) : real(0);
  const real dt = real(dtd);
  const real one = real(1);
  // face indices of this node's x-line and y-line
  const int ixR = m.bcx == 0 ? (ix + 1) % m.nx : ix + 1;
  real cRx = (one - a) * P.tb.gR[p] + (p == N ? a * P.tb.invw[N] : real(0));
  real cLx = (one - a) * P.tb.gL[p] - (p == 0 ? a * P.tb.invw[0] : real(0));
  const size_t nXf = (size_t)m.ny * m.nfx * NFN;
  double unew[M];
#pragma unroll
  for (int v = 0; v < M; ++v) {
    const real FxL = P.b.fx[v * nXf + ((size_t)iy * m.nfx + ix) * NFN + q];
    const real FxR = P.b.fx[v * nXf + ((size_t)iy * m.nfx + ixR) * NFN + q];
    real val = P.b.P[((size_t)v * m.ne + ee) * NP + k] - dt * real(m.invdx) * (FxR * cRx + FxL * cLx);
    if (DIM == 2) {
      const int iyT = m.bcy == 0 ? (iy + 1) % m.ny : iy + 1;
      const size_t nYf = (size_t)m.nfy * m.nx * n;
      const real cRy = (one - a) * P.tb.gR[q] + (q == N ? a * P.tb.invw[N] : real(0));
      const real cLy = (one - a) * P.tb.gL[q] - (q == 0 ? a * P.tb.invw[0] : real(0));
      const real GB = P.b.fy[v * nYf + ((size_t)iy * m.nx + ix) * n + p];
      const real GT = P.b.fy[v * nYf + ((size_t)iyT * m.nx + ix) * n + p];
      val -= dt * real(m.invdy) * (GT * cRy + GB * cLy);
    }
    unew[v] = double(val);
    ATU(v, k) = unew[v];
  }
  __syncthreads();

  // element mean: FP64 sum in FP64 mode; in FP32_BULK mode the conservative
  // FP64 mean update of eq. (upmean) (plus the source mean), and the nodes are
  // re-centred on it
  for (int v = k; v < M; v += NP) {
    double mean;
    if constexpr (MIXED) {
      double fxs = 0.0, fys = 0.0;
      for (int j = 0; j < NFN; ++j) {
        const double wj = DIM == 2 ? td.w[j] : 1.0;
        fxs += wj * (double(P.b.fx[v * nXf + ((size_t)iy * m.nfx + ixR) * NFN + j]) -
                     double(P.b.fx[v * nXf + ((size_t)iy * m.nfx + ix) * NFN + j]));
      }
      if (DIM == 2) {
        const int iyT = m.bcy == 0 ? (iy + 1) % m.ny : iy + 1;
        const size_t nYf = (size_t)m.nfy * m.nx * n;
        for (int j = 0; j < n; ++j)
          fys += td.w[j] * (double(P.b.fy[v * nYf + ((size_t)iyT * m.nx + ix) * n + j]) -
                            double(P.b.fy[v * nYf + ((size_t)iy * m.nx + ix) * n + j]));
      }
      mean = P.b.umean[(size_t)v * m.ne + ee] + dtd * P.b.smean[(size_t)v * m.ne + ee] -
             dtd * m.invdx * fxs - (DIM == 2 ? dtd * m.invdy * fys : 0.0);
      double m32 = 0.0;
      for (int kk = 0; kk < NP; ++kk) {
        const int pp = DIM == 2 ? kk % n : kk, qq = DIM == 2 ? kk / n : 0;
        m32 += (DIM == 2 ? td.w[pp] * td.w[qq] : td.w[pp]) * ATU(v, kk);
      }
      sShift[el * M + v] = mean - m32;  // shift that re-centres the nodes
    } else {
      mean = 0.0;
      for (int kk = 0; kk < NP; ++kk) {
        const int pp = DIM == 2 ? kk % n : kk, qq = DIM == 2 ? kk / n : 0;
        mean += (DIM == 2 ? td.w[pp] * td.w[qq] : td.w[pp]) * ATU(v, kk);
      }
    }
    sMean[el * M + v] = mean;
  }
  __syncthreads();
  double ubar[M];
#pragma unroll
  for (int v = 0; v < M; ++v) ubar[v] = sMean[el * M + v];
  if constexpr (MIXED) {
    double shift[M];
#pragma unroll
    for (int v = 0; v < M; ++v) shift[v] = sShift[el * M + v];
    __syncthreads();
#pragma unroll
    for (int v = 0; v < M; ++v) {
      unew[v] += shift[v];
      ATU(v, k) = unew[v];
    }
    __syncthreads();
  }

  // ---------------- positivity scaling limiter (FP64 theta) --------------
  int bad = 0;
  const bool mean_ok = admissible<EQ>(ubar, m);
  if (EQ::K > 0 && !mean_ok) bad |= kStInadmissible;
  const bool do_scale = (m.limiter & kLimScaling) && EQ::K > 0;
  const bool traces = (m.limiter & kLimTraces) != 0;
  double pts[1 + SPT][M];
  int npt = 1;
#pragma unroll
  for (int v = 0; v < M; ++v) pts[0][v] = unew[v];
  if (do_scale && traces) {
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
          pts[npt][v] = acc;
        }
        ++npt;
      }
    }
  }
  if (do_scale) {
    // density: theta1 from the smallest density over the checked points
    double rmin = pts[0][0];
    for (int t = 1; t < npt; ++t) rmin = fmin(rmin, pts[t][0]);
    sRed[el * NP + k] = rmin;
    __syncthreads();
    if (k == 0) {
      double r = sRed[el * NP];
      for (int kk = 1; kk < NP; ++kk) r = fmin(r, sRed[el * NP + kk]);
      const double eps1 = fmin(1e-12, ubar[0]);
      sTh[el] = (mean_ok && r < eps1) ? (ubar[0] - eps1) / (ubar[0] - r) : 2.0;  // 2: untouched
    }
    __syncthreads();
    const double th1 = sTh[el];
    if (th1 <= 1.0)
      for (int t = 0; t < npt; ++t) pts[t][0] = ubar[0] + th1 * (pts[t][0] - ubar[0]);
    // second constraint: bisection along the segment from the mean
    const double eps2 = fmin(1e-12, EQ::constraint(ubar, 1, m));
    double tmin = 1.0;
    if (mean_ok)
      for (int t = 0; t < npt; ++t) {
        if (EQ::constraint(pts[t], 1, m) >= eps2) continue;
        double lo = 0.0, hi = 1.0, tmp[M];
        for (int it = 0; it < 50; ++it) {
          const double mid = 0.5 * (lo + hi);
#pragma unroll
          for (int v = 0; v < M; ++v) tmp[v] = ubar[v] + mid * (pts[t][v] - ubar[v]);
          if (EQ::constraint(tmp, 1, m) >= eps2) lo = mid;
          else hi = mid;
        }
        tmin = fmin(tmin, lo);
      }
    __syncthreads();
    sRed[el * NP + k] = tmin;
    __syncthreads();
    if (k == 0) {
      double r = sRed[el * NP];
      for (int kk = 1; kk < NP; ++kk) r = fmin(r, sRed[el * NP + kk]);
      sTh[el] = r;
    }
    __syncthreads();
    const double th2 = sTh[el];
    if (th2 < 1.0)
      for (int t = 0; t < npt; ++t)
#pragma unroll
        for (int v = 0; v < M; ++v) pts[t][v] = ubar[v] + th2 * (pts[t][v] - ubar[v]);
#pragma unroll
    for (int v = 0; v < M; ++v) unew[v] = pts[0][v];
    if (mean_ok)
      for (int t = 0; t < npt; ++t)
        if (!admissible<EQ>(pts[t], m)) bad |= kStInadmissible;
  }
#pragma unroll
  for (int v = 0; v < M; ++v)
    if (!isfinite(unew[v])) bad |= kStNonFinite;
  if (valid && bad) {
    atomicOr(&P.b.ctl->status, bad);
    atomicMin(&P.b.ctl->bad_elem, e);
  }
  if (valid) {
#pragma unroll
    for (int v = 0; v < M; ++v) {
      const size_t gi = ((size_t)v * m.ne + e) * NP + k;
      if constexpr (MIXED) P.b.u[gi] = real(unew[v] - ubar[v]);
      else P.b.u[gi] = real(unew[v]);
    }
    if constexpr (MIXED) {
      for (int v = k; v < M; v += NP) P.b.umean[(size_t)v * m.ne + e] = ubar[v];
    }
  }

  // ---------------- indicator of the new state and the CFL rate ---------
  if ((m.limiter & kLimBlend) && m.alpha_mode == 0) {
    __syncthreads();
    sRed[el * NP + k] = EQ::indicator_var(unew, m);
    __syncthreads();
    double al = 0.0;
    indicator_alpha<DIM, N>(m, td, sRed, sT, el, k, &al);
    if (valid && k == 0) P.b.alpha_raw[e] = al;
  }
  __syncthreads();
  if (k == 0) {
    double r = EQ::speed(ubar, 0, m) * m.invdx;
    if (DIM == 2) r += EQ::speed(ubar, 1, m) * m.invdy;
    sTh[el] = valid ? r : 0.0;
  }
  __syncthreads();
  double brate = 0.0;
  if (tid == 0)
    for (int j = 0; j < epb; ++j) brate = fmax(brate, sTh[j]);
  finish_block(P.b.ctl, brate, 1, dtd, last_step);
#undef ATU
}

// ===========================================================================
// After cr_set_state: validate the input, compute the indicator of the state
// and the CFL rate of eq. (time.step.2d) (no time advance).
template <int DIM, int N, class EQ, typename real, bool MIXED>
__global__ void k_prologue(const KParams<real> P) {
  constexpr int n = N + 1;
  constexpr int NP = DIM == 2 ? n * n : n;
  constexpr int M = EQ::M;
  const Mesh& m = P.m;
  const Tab<double>& td = P.td;
  const int epb = blockDim.x / NP;
  const int tid = threadIdx.x;
  const int el = tid / NP, k = tid - el * NP;
  const int e = blockIdx.x * epb + el;
  const bool valid = e < m.ne;
  const int ee = valid ? e : m.ne - 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sU = reinterpret_cast<double*>(smem_raw);  // [M][epb][NP]
  double* sRed = sU + M * epb * NP;
  double* sT = sRed + epb * NP;
  double* sMean = sT + epb * NP;
  double* sTh = sMean + 2 * epb * M;
  const int stride = epb * NP;
  double u[M];
  int bad = 0;
#pragma unroll
  for (int v = 0; v < M; ++v) {
    u[v] = double(P.b.u[((size_t)v * m.ne + ee) * NP + k]);
    if constexpr (MIXED) u[v] += P.b.umean[(size_t)v * m.ne + ee];
    sU[v * stride + el * NP + k] = u[v];
    if (!isfinite(u[v])) bad = kStInvalidInput;
  }
  if (!admissible<EQ>(u, m)) bad = kStInvalidInput;
  if (valid && bad) {
    atomicOr(&P.b.ctl->status, bad);
    atomicMin(&P.b.ctl->bad_elem, e);
  }
  __syncthreads();
  for (int v = k; v < M; v += NP) {
    double mean = 0.0;
    for (int kk = 0; kk < NP; ++kk) {
      const int pp = DIM == 2 ? kk % n : kk, qq = DIM == 2 ? kk / n : 0;
      mean += (DIM == 2 ? td.w[pp] * td.w[qq] : td.w[pp]) * sU[v * stride + el * NP + kk];
    }
    sMean[el * M + v] = mean;
  }
  __syncthreads();
  if ((m.limiter & kLimBlend) && m.alpha_mode == 0) {
    sRed[el * NP + k] = EQ::indicator_var(u, m);
    __syncthreads();
    double al = 0.0;
    indicator_alpha<DIM, N>(m, td, sRed, sT, el, k, &al);
    if (valid && k == 0) P.b.alpha_raw[e] = al;
  }
  __syncthreads();
  if (k == 0) {
    double ubar[M];
#pragma unroll
    for (int v = 0; v < M; ++v) ubar[v] = sMean[el * M + v];
    double r = EQ::speed(ubar, 0, m) * m.invdx;
    if (DIM == 2) r += EQ::speed(ubar, 1, m) * m.invdy;
    sTh[el] = valid ? r : 0.0;
  }
  __syncthreads();
  double brate = 0.0;
  if (tid == 0)
    for (int j = 0; j < epb; ++j) brate = fmax(brate, sTh[j]);
  finish_block(P.b.ctl, brate, 0, 0.0, 0);
}

// FP32_BULK state conversion: FP64 nodal values <-> FP64 mean + FP32 fluctuation.
template <int DIM, int N, int M>
__global__ void k_split_state(const double* __restrict__ in, float* __restrict__ fl,
                              double* __restrict__ mean, int ne, Tab<double> td) {
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
  for (int kk = 0; kk < NP; ++kk) fl[(size_t)idx * NP + kk] = float(x[kk] - mu);
}

template <int NP>
__global__ void k_join_state(const float* __restrict__ fl, const double* __restrict__ mean,
                             double* __restrict__ out, int nvals) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // one thread per value
  if (idx >= nvals) return;
  out[idx] = mean[idx / NP] + double(fl[idx]);
}

}  // namespace crk
