// Fused face + cell passes of the Schur-complement vmult, the Schur
// right-hand side and the velocity recovery (Section 3: the B, C and
// implicit Rusanov face terms are evaluated inside the cell kernels).
//
// A block owns EPB cells.  It evaluates the numerical fluxes at every face
// point of its own cells itself and keeps the lift values in shared memory,
// so no face flux goes through global memory and no separate face kernel
// runs.  The block's threads form N groups of EPB x N^(d-1) threads; group
// g takes the faces f = g mod N, each thread one point (cell c, point t) of
// them, so that the face index is a compile-time constant in the unrolled
// face loop.  The plus-side value at a conforming (or periodic) face point
// comes either
//   STAGE = true : from the neighbour cell's node line through that point,
//                  read by the thread itself (mostly L2 hits: the vectors
//                  are a few tens of MB) and contracted to the face, or
//   STAGE = false: from a per-slot trace array written by k_trace, which
//                  spends no arithmetic on the neighbour's trace (the
//                  choice where the FP64 pipe binds).
// Both sides of a face evaluate the same flux with their own outward normal
// (exact negatives of each other), so every face term stays conservative.
// Faces on a 2:1 interface (fine or coarse side, cell face code -2) take
// their lift values from the slot array, filled by the face kernels and the
// mortar gather run on the hanging face points only.
#pragma once

#include "ops.cuh"

namespace dg {

template <int DIM, int N>
struct FusedShape {
  static constexpr int NP = ipow(N, DIM), NFP = ipow(N, DIM - 1), NF = 2 * DIM, NSL = NF * NFP;
  static constexpr int EPB = NP >= 256 ? 1 : 256 / NP;
  static constexpr int THREADS = EPB * NP;
};

// resident blocks per SM each precision asks the register allocator for:
// the FP32 kernels wait on barriers and loads, not on a pipe, so more warps
// hide more latency; the FP64 ones are bound by the FP64 pipe and the pair
// ones would spill below 64 registers
template <typename T>
struct FusedOcc {
  static constexpr int MIN_BLOCKS = std::is_same<T, float>::value ? 5 : 4;
};

// node line of face f's point t: first node and stride along the normal
template <int DIM, int N>
__device__ __forceinline__ void face_line(int f, int t, int& base, int& stride) {
  const int a = f >> 1;
  int idx[3] = {0, 0, 0};
#pragma unroll
  for (int b = 0, rr = t; b < DIM; ++b) {
    if (b == a) continue;
    idx[b] = rr % N;
    rr /= N;
  }
  stride = a == 0 ? 1 : (a == 1 ? N : N * N);
  base = idx[0] + N * idx[1] + N * N * idx[2];
}

// Outward n dS of face f of cell e at its point t: loaded from the per-slot
// array, or (snS == null, FP32 only) recomputed from the cell's corner offsets:
// n dS = (+-1) w_t C_a(xi), C_a the cofactor row of the normal direction a
// at xi_a = s and the tangential Gauss-Legendre nodes, w_t the product of
// the tangential weights.
template <typename T, int DIM, int N>
__device__ __forceinline__ void slot_normal(const CellGeo<T>& g, const T* __restrict__ snS, int64_t S,
                                            int64_t e, int f, int t, int64_t sl, const T* sxw, T nS[DIM],
                                            const T* tcs = nullptr) {
  if (!std::is_same<T, float>::value || snS) {   // FP64 always loads
#pragma unroll
    for (int b = 0; b < DIM; ++b) nS[b] = __ldg(snS + b * S + sl);
    return;
  }
  const int a = f >> 1, s = f & 1;
  T xi[3] = {0, 0, 0}, wt = 1;
  xi[a] = (T)s;
#pragma unroll
  for (int b = 0, rr = t; b < DIM; ++b) {
    if (b == a) continue;
    xi[b] = sxw[rr % N];
    wt *= sxw[N + rr % N];
    rr /= N;
  }
  T C[DIM][DIM], det;
  if (tcs)
    terrain_row<T, DIM>(tcs, xi, C, det);
  else
    corner_cofactors<T, DIM>(g.lv + e * (DIM << DIM), g.terrain, xi, C, det);
  const T sw = (s ? (T)1 : (T)-1) * wt;
#pragma unroll
  for (int b = 0; b < DIM; ++b) nS[b] = sw * C[a][b];
}

// lift of NFLD fields from the block's shared lift values (field stride NSL)
template <typename T, int DIM, int N, int NFLD, typename TB>
__device__ __forceinline__ void lift_shared(const TB& tb, const T* sl, const int idx[3], T* r) {
  constexpr int NFP = ipow(N, DIM - 1), NF = 2 * DIM, NSL = NF * NFP;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int a = f >> 1, s = f & 1;
    const T Lv = tb.L[s][idx[a]];
    const int k = f * NFP + tang_index<DIM, N>(idx, a);
#pragma unroll
    for (int q = 0; q < NFLD; ++q) r[q] -= sl[q * NSL + k] * Lv;
  }
}

// Gauss-Legendre nodes and weights of the block in shared memory (for the
// recomputed metric and normals)
template <typename T, int N>
__device__ __forceinline__ void stage_nodes_all(const CellGeo<T>& g, T* sxw) {
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      sxw[k] = g.x[k];
      sxw[N + k] = g.w[k];
    }
  }
}

// FP32 terrain-following meshes: the block's cells' 16 terrain coefficients
// in shared memory (the metric and the normals are recomputed from them)
template <typename T, int EPB>
__device__ __forceinline__ void stage_terrain(const CellGeo<T>& g, int64_t e0, int64_t E, T (*stc)[16]) {
  if (std::is_same<T, float>::value && g.tc) {
    for (int k = threadIdx.x; k < EPB * 16; k += blockDim.x) {
      const int c = k / 16, j = k % 16;
      stc[c][j] = e0 + c < E ? __ldg(g.tc + (e0 + c) * 16 + j) : (T)0;
    }
  }
}

// Gradient pass: weak gradient G = M^{-1}[-int x grad(phi) + int {x} phi.n]
// with centred face values, and the implicit Rusanov jump; then
//  VMULT  : w = rho^{-1} (I + beta J)^{-1} G (R2) or G / rho (R1) -> wv (DIM
//           spatial comps); y = x + pen - (gamma-1) a_dt^2 g G_z (R2)
//  RECOVER: u = ustar - a_dt w (3 comps; no penalty)
template <typename T, int DIM, int N, int MODE, bool STAGE>
__global__ void __launch_bounds__(FusedShape<DIM, N>::THREADS, FusedOcc<T>::MIN_BLOCKS)
k_grad_fused(const T* __restrict__ x, const T* __restrict__ tx, const int* __restrict__ cface,
             const T* __restrict__ snS, const T* __restrict__ pcs, const T* __restrict__ irho, CellGeo<T> geo,
             const T* __restrict__ slot, int64_t E, int64_t S, Tables<T> tb, ImplK ph, T* __restrict__ wv,
             T* __restrict__ y, const T* __restrict__ ustar, T* __restrict__ uout) {
  using FS = FusedShape<DIM, N>;
  constexpr int NP = FS::NP, EPB = FS::EPB, NF = FS::NF, NFP = FS::NFP, NSL = FS::NSL;
  __shared__ T sx[EPB][NP];
  __shared__ T sxp[EPB][NSL];     // plus-side values at the block's face points
  __shared__ T slf[EPB][DIM + 1][NSL];
  __shared__ T sm[EPB][DIM][DIM][NP];
  __shared__ T sxw[2 * N];
  __shared__ T stc[std::is_same<T, float>::value ? EPB : 1][16];
  __shared__ SharedTables<T, N> stb;
  const int le = threadIdx.x / NP, i = threadIdx.x % NP;
  const int64_t e0 = (int64_t)blockIdx.x * EPB;
  const int64_t e = e0 + le;
  const bool active = e < E;
  const int64_t Nn = E * NP;
  const int64_t node = active ? e * NP + i : 0;
  const bool tcell = std::is_same<T, float>::value && geo.tc != nullptr;
  stage_terrain<T, EPB>(geo, e0, E, stc);
  stage_tables<T, N>(tb, stb);
  int idx[3];
  node_index<DIM, N>(i, idx);
  const T xv = active ? __ldg(x + node) : (T)0;
  sx[le][i] = xv;
  // face points: thread group grp takes the faces f = grp mod N; its
  // global reads (face codes, the neighbour's node line or its trace, the
  // penalty coefficient) are issued before the block's first barrier
  constexpr int GS = EPB * NFP;
  const int grp = threadIdx.x / GS, cc = (threadIdx.x % GS) / NFP, tt = threadIdx.x % NFP;
  const int64_t ec = e0 + cc;
  int codes[NF];
  T pen[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    codes[f] = -1;
    pen[f] = 0;
    if (f % N != grp || ec >= E) continue;
    const int code = __ldg(cface + ec * NF + f);
    codes[f] = code;
    const int64_t sl = ec * NSL + f * NFP + tt;
    T xp = 0;
    if (code >= 0) {
      if (STAGE) {
        int base, stride;
        face_line<DIM, N>(f, tt, base, stride);
        const T* __restrict__ nb = x + (int64_t)code * NP + base;
#pragma unroll
        for (int j = 0; j < N; ++j) xp += tb.L[(f & 1) ^ 1][j] * __ldg(nb + j * stride);   // compile-time indices
      } else {
        xp = __ldg(tx + ((int64_t)code * NF + (f ^ 1)) * NFP + tt);
      }
      if (pcs) pen[f] = __ldg(pcs + sl);
    } else if (code == -3 && pcs) {
      pen[f] = __ldg(pcs + sl);
    }
    sxp[cc][f * NFP + tt] = xp;
  }
  stage_nodes_all<T, N>(geo, sxw);
  __syncthreads();
  // numerical fluxes at the face points (own traces from the staged cell)
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    if (f % N != grp || ec >= E) continue;
    const int code = codes[f];
    const int r = f * NFP + tt;
    const int64_t sl = ec * NSL + r;
    if (code == -2) {
#pragma unroll
      for (int q = 0; q <= DIM; ++q) slf[cc][q][r] = __ldg(slot + q * S + sl);
      continue;
    }
    T xm = 0;
    if (STAGE) {
      int base, stride;
      face_line<DIM, N>(f, tt, base, stride);
#pragma unroll
      for (int j = 0; j < N; ++j) xm += stb.L[f & 1][j] * sx[cc][base + j * stride];
    } else {
      xm = __ldg(tx + sl);
    }
    // wall (-1): {x} = x-, no jump; far field (-3): the linear part, the
    // outer state's value is known data of the right-hand side (zero here)
    const T xp = code == -1 ? xm : sxp[cc][r];
    const T avg = code == -1 ? xm : (T)0.5 * (xm + xp);
    T nS[DIM];
    slot_normal<T, DIM, N>(geo, snS, S, ec, f, tt, sl, sxw, nS, tcell ? stc[cc] : nullptr);
#pragma unroll
    for (int b = 0; b < DIM; ++b) slf[cc][b][r] = -avg * nS[b];
    slf[cc][DIM][r] = code == -1 ? (T)0 : -pen[f] * (xm - xp);
  }
  // volume terms: every flux component -x K_ab staged at once, one barrier
  T K[DIM][DIM], iM = 0;
  if (active) node_metric<T, DIM, N>(geo, e, node, Nn, idx, K, iM, sxw, tcell ? stc[le] : nullptr);
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    const int msk = amask_of<DIM>(geo.terrain, b);
#pragma unroll
    for (int a = 0; a < DIM; ++a)
      if ((msk >> a) & 1) sm[le][b][a][i] = active ? -xv * K[a][b] : (T)0;
  }
  __syncthreads();
  T r[DIM + 1];
#pragma unroll
  for (int b = 0; b < DIM; ++b) r[b] = contract<T, DIM, N>(stb, sm[le][b], i, idx, amask_of<DIM>(geo.terrain, b));
  r[DIM] = 0;
  if (!active) return;
  lift_shared<T, DIM, N, DIM + 1>(stb, &slf[le][0][0], idx, r);
  T G[3] = {0, 0, 0};
#pragma unroll
  for (int b = 0; b < DIM; ++b) G[comp_of<DIM>(b)] = iM * r[b];
  const T ir = __ldg(irho + node);
  T w[3];
  if (ph.r2) {
    const T beta = beta_of<T>(ph, e);
    const T d = (ph.fcell || ph.fcell32) ? (T)1 / (1 + beta * beta) : kp<T>(ph.dbeta, ph.dbeta_f, ph.dbeta_p);
    w[0] = (G[0] + beta * G[1]) * d * ir;
    w[1] = (G[1] - beta * G[0]) * d * ir;
    w[2] = G[2] * ir;
  } else {
    w[0] = G[0] * ir;
    w[1] = G[1] * ir;
    w[2] = G[2] * ir;
  }
  if (MODE == GRAD_VMULT) {
#pragma unroll
    for (int b = 0; b < DIM; ++b) wv[b * Nn + node] = w[comp_of<DIM>(b)];
    T yv = xv + iM * r[DIM];
    if (ph.r2) yv -= kp<T>(ph.cgrav, ph.cgrav_f, ph.cgrav_p) * G[2];
    y[node] = yv;
  } else {
    const T adt = kp<T>(ph.a_dt, ph.adt_f, ph.adt_p);
#pragma unroll
    for (int c = 0; c < 3; ++c) uout[c * Nn + node] = __ldg(ustar + c * Nn + node) - adt * w[c];
  }
}

// Divergence pass: Div = M^{-1}[-int h rho w . grad(psi) + centred face
// flux {h rho w}.n dS (zero on walls)], h rho = gamma p_lag / (gamma - 1),
// its face values from the per-slot traces trh; then
//  VMULT: y -= (gamma-1) a_dt^2 Div
//  RHS  : y = (gamma-1) [e_hat - rho |u_lag|^2 / 2 - a_dt (Div + g rho w3_z)],
//         w3_z = ustar_z (R2) or u_lag_z (R1)
template <typename T, int DIM, int N, int MODE, bool STAGE>
__global__ void __launch_bounds__(FusedShape<DIM, N>::THREADS, FusedOcc<T>::MIN_BLOCKS)
k_div_fused(Fields<T> wv, const T* __restrict__ tw, const T* __restrict__ trh, const int* __restrict__ cface,
            const T* __restrict__ snS, const T* __restrict__ plag, CellGeo<T> geo, const T* __restrict__ slot,
            int64_t E, int64_t S, Tables<T> tb, ImplK ph, T* __restrict__ y, const T* __restrict__ ehat,
            const T* __restrict__ rho, const T* __restrict__ ulag, const T* __restrict__ ustar) {
  using FS = FusedShape<DIM, N>;
  constexpr int NP = FS::NP, EPB = FS::EPB, NF = FS::NF, NFP = FS::NFP, NSL = FS::NSL;
  __shared__ T sw[EPB][DIM][NP];
  __shared__ T swp[EPB][DIM][NSL];   // plus-side w components at the block's face points
  __shared__ T slf[EPB][NSL];
  __shared__ T sm[EPB][DIM][NP];
  __shared__ T sxw[2 * N];
  __shared__ T stc[std::is_same<T, float>::value ? EPB : 1][16];
  __shared__ SharedTables<T, N> stb;
  const int le = threadIdx.x / NP, i = threadIdx.x % NP;
  const int64_t e0 = (int64_t)blockIdx.x * EPB;
  const int64_t e = e0 + le;
  const bool active = e < E;
  const int64_t Nn = E * NP;
  const int64_t node = active ? e * NP + i : 0;
  const bool tcell = std::is_same<T, float>::value && geo.tc != nullptr;
  stage_terrain<T, EPB>(geo, e0, E, stc);
  stage_tables<T, N>(tb, stb);
  int idx[3];
  node_index<DIM, N>(i, idx);
  const T gam = kp<T>(ph.gamma, ph.gamma_f, ph.gamma_p);
  const T gm1 = gam - 1;
  T wl[DIM];
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    wl[b] = active ? __ldg(wv.f[b] + node) : (T)0;
    sw[le][b][i] = wl[b];
  }
  // face points: thread group grp takes the faces f = grp mod N (see above);
  // the global reads (codes, h rho traces, the neighbour's w) go first
  constexpr int GS = EPB * NFP;
  const int grp = threadIdx.x / GS, cc = (threadIdx.x % GS) / NFP, tt = threadIdx.x % NFP;
  const int64_t ec = e0 + cc;
  int codes[NF];
  T hm[NF], hp[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    codes[f] = -1;
    hm[f] = hp[f] = 0;
    if (f % N != grp || ec >= E) continue;
    const int code = __ldg(cface + ec * NF + f);
    codes[f] = code;
    const int64_t sl = ec * NSL + f * NFP + tt;
    if (code >= 0 || code == -3) hm[f] = __ldg(trh + sl);
    if (code < 0) continue;
    const int64_t sp = ((int64_t)code * NF + (f ^ 1)) * NFP + tt;
    hp[f] = __ldg(trh + sp);
    int base, stride;
    face_line<DIM, N>(f, tt, base, stride);
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      T wp = 0;
      if (STAGE) {
        const T* __restrict__ nb = wv.f[b] + (int64_t)code * NP + base;
#pragma unroll
        for (int j = 0; j < N; ++j) wp += tb.L[(f & 1) ^ 1][j] * __ldg(nb + j * stride);   // compile-time indices
      } else {
        wp = __ldg(tw + b * S + sp);
      }
      swp[cc][b][f * NFP + tt] = wp;
    }
  }
  stage_nodes_all<T, N>(geo, sxw);
  __syncthreads();
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    if (f % N != grp || ec >= E) continue;
    const int code = codes[f];
    const int r = f * NFP + tt;
    const int64_t sl = ec * NSL + r;
    if (code == -2) {
      slf[cc][r] = __ldg(slot + sl);
      continue;
    }
    if (code == -1) {   // wall: the mirror velocity makes {h rho w}.n vanish
      slf[cc][r] = 0;
      continue;
    }
    T nS[DIM];
    slot_normal<T, DIM, N>(geo, snS, S, ec, f, tt, sl, sxw, nS, tcell ? stc[cc] : nullptr);
    int base, stride;
    face_line<DIM, N>(f, tt, base, stride);
    // own normal flux (w-.n dS) and, on a conforming face, the neighbour's
    // (w+.n dS); far field (-3): the linear part (h rho w)-.n / 2 only
    T fm = 0, fp = 0;
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      T wm = 0;
      if (STAGE) {
#pragma unroll
        for (int j = 0; j < N; ++j) wm += stb.L[f & 1][j] * sw[cc][b][base + j * stride];
      } else {
        wm = __ldg(tw + b * S + sl);
      }
      fm += wm * nS[b];
      if (code >= 0) fp += swp[cc][b][r] * nS[b];
    }
    slf[cc][r] = -(T)0.5 * (hm[f] * fm + hp[f] * fp);
  }
  T iM = 0;
  if (active) {
    T K[DIM][DIM];
    node_metric<T, DIM, N>(geo, e, node, Nn, idx, K, iM, sxw, tcell ? stc[le] : nullptr);
    const T hr = gam / gm1 * __ldg(plag + node);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      T v = 0;
#pragma unroll
      for (int b = 0; b < DIM; ++b)
        if (!(geo.terrain && kzero<DIM>(a, b))) v += K[a][b] * wl[b];
      sm[le][a][i] = -hr * v;
    }
  } else {
#pragma unroll
    for (int a = 0; a < DIM; ++a) sm[le][a][i] = 0;
  }
  __syncthreads();
  T r[1];
  r[0] = contract<T, DIM, N>(stb, sm[le], i, idx);
  if (!active) return;
  lift_shared<T, DIM, N, 1>(stb, &slf[le][0], idx, r);
  const T div = iM * r[0];
  const T adt = kp<T>(ph.a_dt, ph.adt_f, ph.adt_p);
  if (MODE == DIV_VMULT) {
    y[node] -= gm1 * adt * adt * div;
  } else {
    const T rh = __ldg(rho + node);
    T u2 = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T uc = __ldg(ulag + c * Nn + node);
      u2 += uc * uc;
    }
    const T wz = ph.r2 ? __ldg(ustar + 2 * Nn + node) : __ldg(ulag + 2 * Nn + node);
    y[node] = gm1 * (__ldg(ehat + node) - (T)0.5 * rh * u2 - adt * (div + kp<T>(ph.g, ph.g_f, ph.g_p) * rh * wz));
  }
}

// implicit Rusanov coefficient of every face point, copied to both of its
// own slots (conforming and periodic faces; the others do not read it)
template <typename T>
__global__ void k_pcoef_slots(const int* __restrict__ fp_minus, const int* __restrict__ fp_plus,
                              const int* __restrict__ fp_far, const T* __restrict__ pcoef, int64_t nF,
                              T* __restrict__ pcs) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= nF) return;
  const int code = fp_plus[p];
  const bool far = code == -1 && fp_far && fp_far[p] >= 0;
  if (code < 0 && !far) return;
  const T v = pcoef[p];
  pcs[fp_minus[p]] = v;
  if (code >= 0) pcs[code] = v;
}

// Outer data of the far-field faces in the stage system (reading of the
// non-reflecting top, Section 4.3): with the outer state known, the halves
// of B p, C u and the implicit Rusanov term that it carries move to the
// right-hand sides, b_far = a_dt int_far (p_far / 2) n . phi_i and g_far =
// a_dt int_far (h rho u)_far . n / 2 psi_i - a_dt / (2 (gamma - 1))
// int_far lambda p_far psi_i.  As nodal predictors: m_hat -= M^{-1} b_far,
// e_hat -= M^{-1} g_far (eh may be null: the recovery needs m_hat only).
// One thread per far point of face type f (a line of nodes normal to a face
// belongs to one point of it, so a launch writes every node at most once).
template <typename T, int DIM, int N>
__global__ void k_far_affine(FaceTopo ft, const int* __restrict__ far_p, int64_t g0, int64_t g1, int f,
                             const T* __restrict__ invM, const T* __restrict__ pcoef, ImplK ph, Tables<T> tb,
                             T* __restrict__ mh, T* __restrict__ eh, int64_t Nn) {
  constexpr int NP = ipow(N, DIM), NFP = ipow(N, DIM - 1), NSL = 2 * DIM * NFP;
  const int64_t g = g0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= g1) return;
  const int64_t p = __ldg(far_p + g);
  const int sm = __ldg(ft.fp_minus + p);
  const int64_t e = sm / NSL;
  const int t = (sm % NSL) % NFP;
  const T* fq = far_ptr<T>(ft);
  const T gam = kp<T>(ph.gamma, ph.gamma_f, ph.gamma_p), adt = kp<T>(ph.a_dt, ph.adt_f, ph.adt_p);
  const T rf = __ldg(fq + g);
  T uf[3], mu = 0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T mc = __ldg(fq + (1 + c) * ft.nFar + g);
    uf[c] = mc / rf;
    mu += mc * uf[c];
  }
  const T pf = (gam - 1) * (__ldg(fq + 4 * ft.nFar + g) - (T)0.5 * mu);
  T vb[DIM], unS = 0;
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    const T n = __ldg(geo_ptr<T>(ft) + b * ft.nF + p);
    vb[b] = adt * (T)0.5 * pf * n;
    unS += uf[comp_of<DIM>(b)] * n;
  }
  T ve = adt * (T)0.5 * gam / (gam - 1) * pf * unS;
  if (ph.penalty && pcoef) ve -= __ldg(pcoef + p) * pf / (gam - 1);
  const int s = f & 1;
  int base, stride;
  face_line<DIM, N>(f, t, base, stride);
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int64_t node = e * NP + base + k * stride;
    const T w = __ldg(invM + node) * tb.L[s][k];
#pragma unroll
    for (int b = 0; b < DIM; ++b) mh[comp_of<DIM>(b) * Nn + node] -= w * vb[b];
    if (eh) eh[node] -= w * ve;
  }
}

}  // namespace dg
