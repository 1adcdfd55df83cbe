// Operator kernels of libdgimex: face traces, numerical fluxes, 2:1 mortar
// gather, sum-factorised cell kernels of the explicit operator and of the
// Schur-complement vmult.  Templated on the scalar type T and on the
// compile-time (DIM, N = r + 1).
//
// Face-slot convention.  Every cell owns 2*DIM faces x N^(DIM-1) face
// points ("slots", slot = (e * 2 DIM + f) * NFP + pt, face f = 2a + s at
// xi_a = s, face points in tangential tensor order).  A face kernel writes
// into each slot the value v such that the cell's weak residual receives
// -v * l_{i_a}(s) at node i (the lift).  Every slot is written exactly once
// per pass (interior side, wall, fine hanging side, or the coarse gather),
// so no slot buffer is ever cleared and no atomics are used.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace dg {

// face geometry (n dS) in the kernel's precision
template <typename T> __device__ __forceinline__ const T* geo_ptr(const FaceTopo& ft);
template <> __device__ __forceinline__ const double* geo_ptr<double>(const FaceTopo& ft) { return ft.fgeo; }
template <> __device__ __forceinline__ const float* geo_ptr<float>(const FaceTopo& ft) { return ft.fgeo32; }

template <> __device__ __forceinline__ const df64* geo_ptr<df64>(const FaceTopo& ft) { return ft.fgeodf; }

// outer state's traces at the far-field points, in the kernel's precision
// (DG_PAIRS does not run on meshes with far-field faces)
template <typename T> __device__ __forceinline__ const T* far_ptr(const FaceTopo& ft);
template <> __device__ __forceinline__ const double* far_ptr<double>(const FaceTopo& ft) { return ft.far_q; }
template <> __device__ __forceinline__ const float* far_ptr<float>(const FaceTopo& ft) { return ft.far_q32; }
template <> __device__ __forceinline__ const df64* far_ptr<df64>(const FaceTopo& ft) { return ft.far_qdf; }

// far-point index of boundary face point p (-1: slip wall)
__device__ __forceinline__ int far_index(const FaceTopo& ft, int64_t p) {
  return ft.fp_far ? __ldg(ft.fp_far + p) : -1;
}

template <typename T> struct Fields {
  const T* f[5];
  T scale[5];
};

// The 1D tables of a block in shared memory.  Kernel parameters indexed
// with a per-thread index are read through the constant cache one address
// at a time (the ADU pipe bound the first cell kernels); shared memory
// serves a warp's different indices in one pass.
template <typename T, int N>
struct SharedTables {
  T D[N][N];   // D[k][j] = l_j'(xi_k)
  T L[2][N];   // L[s][j] = l_j(s)
};

// one entry per thread (blocks have at least N^2 + 2N threads); a barrier
// must follow before use
template <typename T, int N>
__device__ __forceinline__ void stage_tables(const Tables<T>& tb, SharedTables<T, N>& st) {
  const int k = threadIdx.x;
  if (k < N * N) st.D[k / N][k % N] = tb.D[k / N][k % N];
  else if (k < N * N + 2 * N) st.L[(k - N * N) / N][(k - N * N) % N] = tb.L[(k - N * N) / N][(k - N * N) % N];
}

// tangential index of node i for faces normal to direction a
template <int DIM, int N>
__device__ __forceinline__ int tang_index(const int idx[3], int a) {
  int t = 0, mul = 1;
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    if (b == a) continue;
    t += idx[b] * mul;
    mul *= N;
  }
  return t;
}

template <int DIM, int N>
__device__ __forceinline__ void node_index(int i, int idx[3]) {
  idx[0] = i % N;
  idx[1] = DIM > 1 ? (i / N) % N : 0;
  idx[2] = DIM > 2 ? i / (N * N) : 0;
}

// Value of a coarse-face trace at fine point fp of subface `sub` (2:1).
template <typename T, int DIM, int N>
__device__ __forceinline__ T prolong(const Tables<T>& tb, const T* __restrict__ tr, int sub, int fp) {
  if (DIM == 2) {
    T acc = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) acc += tb.P[sub][fp][j] * tr[j];
    return acc;
  } else {
    int f0 = fp % N, f1 = fp / N, b0 = sub & 1, b1 = sub >> 1;
    T acc = 0;
#pragma unroll
    for (int j1 = 0; j1 < N; ++j1) {
      T row = 0;
#pragma unroll
      for (int j0 = 0; j0 < N; ++j0) row += tb.P[b0][f0][j0] * tr[j0 + N * j1];
      acc += tb.P[b1][f1][j1] * row;
    }
    return acc;
  }
}

template <typename T, int DIM, int N>
__device__ __forceinline__ T prolong_weight(const Tables<T>& tb, int sub, int fp, int j) {
  if (DIM == 2) return tb.P[sub][fp][j];
  return tb.P[sub & 1][fp % N][j % N] * tb.P[sub >> 1][fp / N][j / N];
}

// ---------------------------------------------------------------------------
// traces: slot values of up to 5 nodal fields (times a per-field scale)
//
// A block owns TraceShape::CPB consecutive cells.  Their nodal values of all
// fields are staged in shared memory with coalesced loads (each value is read
// from HBM once), then every slot of those cells, (e * 2d + f) * NFP + t, is
// the 1D interpolation along the face normal of one node line, written with
// coalesced stores (a cell's slots are contiguous).
// ---------------------------------------------------------------------------
template <int DIM, int N>
struct TraceShape {
  static constexpr int NP = ipow(N, DIM), NFP = ipow(N, DIM - 1), NS = 2 * DIM * NFP;
  static constexpr int CPB = NP >= 512 ? 1 : 512 / NP;     // about 512 nodes per block
  static constexpr int THREADS = 256;
};

template <int DIM, int N>
inline unsigned trace_grid(int64_t E) {
  return grid_for(E, TraceShape<DIM, N>::CPB);
}

// slots [0, nc * NS) of the block's cells from the staged values; SCALED
// multiplies each field by its scale (the FP64 pipe bounds this kernel, and
// the multiply is a fifth of its arithmetic, so unit scales skip it)
template <typename T, int DIM, int N, int NFLD, bool SCALED>
__device__ __forceinline__ void trace_slots(const T (*__restrict__ sv)[TraceShape<DIM, N>::CPB * TraceShape<DIM, N>::NP],
                                            const Fields<T>& in, int nc, int64_t out0, T* __restrict__ trc,
                                            int64_t S, const SharedTables<T, N>& tb) {
  using TS = TraceShape<DIM, N>;
  constexpr int NP = TS::NP, NFP = TS::NFP, NS = TS::NS;
  for (int i = threadIdx.x; i < nc * NS; i += TS::THREADS) {
    const int c = i / NS;
    const int r = i - c * NS;
    const int f = r / NFP, pt = r - f * NFP;
    const int a = f >> 1, s = f & 1;
    int idx[3] = {0, 0, 0};
    for (int b = 0, rr = pt; b < DIM; ++b) {
      if (b == a) continue;
      idx[b] = rr % N;
      rr /= N;
    }
    const int stride = a == 0 ? 1 : (a == 1 ? N : N * N);
    const int base = c * NP + idx[0] + N * idx[1] + N * N * idx[2];
#pragma unroll
    for (int q = 0; q < NFLD; ++q) {
      T acc = 0;
#pragma unroll
      for (int k = 0; k < N; ++k) acc += tb.L[s][k] * sv[q][base + k * stride];
      trc[q * S + out0 + i] = SCALED ? acc * in.scale[q] : acc;
    }
  }
}

template <typename T, int DIM, int N, int NFLD>
__global__ void __launch_bounds__(TraceShape<DIM, N>::THREADS)
    k_trace(Fields<T> in, int64_t E, int64_t Nn, T* __restrict__ trc, int64_t S, Tables<T> tb) {
  using TS = TraceShape<DIM, N>;
  constexpr int NP = TS::NP, NS = TS::NS, CPB = TS::CPB;
  __shared__ T sv[NFLD][CPB * NP];
  __shared__ SharedTables<T, N> stb;
  const int64_t e0 = (int64_t)blockIdx.x * CPB;
  const int64_t left = E - e0;
  const int nc = left < CPB ? (int)left : CPB;
  if (nc <= 0) return;
  stage_tables<T, N>(tb, stb);
  bool unit = true;
#pragma unroll
  for (int q = 0; q < NFLD; ++q) {
    unit = unit && in.scale[q] == T(1);
    const T* __restrict__ src = in.f[q] + e0 * NP;
    for (int i = threadIdx.x; i < nc * NP; i += TS::THREADS) sv[q][i] = __ldg(src + i);
  }
  __syncthreads();
  if (unit)
    trace_slots<T, DIM, N, NFLD, false>(sv, in, nc, e0 * NS, trc, S, stb);
  else
    trace_slots<T, DIM, N, NFLD, true>(sv, in, nc, e0 * NS, trc, S, stb);
}

// plus-side value of a traced field at face point p
template <typename T, int DIM, int N>
__device__ __forceinline__ T plus_value(const FaceTopo& ft, const Tables<T>& tb, const T* __restrict__ tr,
                                        int code, T minus_val) {
  if (code >= 0) return __ldg(tr + code);
  if (code == -1) return minus_val;
  int hp = -2 - code;
  int cs = __ldg(ft.hp_cslot + hp), hc = __ldg(ft.hp_code + hp);
  return prolong<T, DIM, N>(tb, tr + cs, hc & 0xff, hc >> 8);
}

// write an antisymmetric face value: minus slot v, plus slot -v, fine
// hanging point -> mortar buffer
template <typename T>
__device__ __forceinline__ void put(T* __restrict__ slot, T* __restrict__ hbuf, int64_t S, int64_t nH,
                                    int fld, int sm, int code, T v) {
  slot[fld * S + sm] = v;
  if (code >= 0) slot[fld * S + code] = -v;
  else if (code <= -2) hbuf[fld * nH + (-2 - code)] = v;
}

// coarse side of 2:1 faces: slot(j) = -sum_sub sum_fp P_sub(fp, j) v(fp)
template <typename T, int DIM, int N, int NFLD>
__global__ void k_hang_gather(FaceTopo ft, const T* __restrict__ hbuf, T* __restrict__ slot,
                              Tables<T> tb) {
  constexpr int NFP = ipow(N, DIM - 1), NSUB = 1 << (DIM - 1);
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ft.nHC * NFP) return;
  int64_t c = t / NFP;
  int j = (int)(t % NFP);
  int cs = ft.hc_slot[c];
#pragma unroll
  for (int q = 0; q < NFLD; ++q) {
    T acc = 0;
    const T* __restrict__ h = hbuf + q * ft.nH + c * NSUB * NFP;
    for (int sub = 0; sub < NSUB; ++sub)
#pragma unroll
      for (int fp = 0; fp < NFP; ++fp) acc += prolong_weight<T, DIM, N>(tb, sub, fp, j) * h[sub * NFP + fp];
    slot[q * ft.S + cs + j] = -acc;
  }
}

// ---------------------------------------------------------------------------
// explicit operator: numerical fluxes at face points
//   slot fields 0..4: non-stiff (rho, m_x, m_y, m_z, E), 5..8: stiff (m_x, m_y, m_z, E)
// ---------------------------------------------------------------------------
template <int DIM> __device__ __forceinline__ int comp_of(int b) { return DIM == 3 ? b : (b == 0 ? 0 : 2); }

template <typename T, int DIM, int N>
__global__ void k_face_explicit(FaceTopo ft, const T* __restrict__ trc, T* __restrict__ slot,
                                T* __restrict__ hbuf, Tables<T> tb, T gamma, T lambda_min) {
  int64_t p = ft.p0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= ft.nF) return;
  const int64_t S = ft.S;
  int sm = __ldg(ft.fp_minus + p), code = __ldg(ft.fp_plus + p);
  T nS[DIM];
  T n2 = 0;
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    nS[b] = __ldg(geo_ptr<T>(ft) + b * ft.nF + p);
    n2 += nS[b] * nS[b];
  }
  T qm[5], qp[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) qm[q] = __ldg(trc + q * S + sm);
  const int g = code == -1 ? far_index(ft, p) : -1;
  if (g >= 0) {
    // far field: the given outer state, in the same fluxes as an interior face
#pragma unroll
    for (int q = 0; q < 5; ++q) qp[q] = __ldg(far_ptr<T>(ft) + q * ft.nFar + g);
  } else if (code == -1) {
    // slip wall: mirror momentum, m+ = m- - 2 (m-.n) n
    T mn = 0;
#pragma unroll
    for (int b = 0; b < DIM; ++b) mn += qm[1 + comp_of<DIM>(b)] * nS[b];
    mn /= n2;
#pragma unroll
    for (int q = 0; q < 5; ++q) qp[q] = qm[q];
#pragma unroll
    for (int b = 0; b < DIM; ++b) qp[1 + comp_of<DIM>(b)] -= 2 * mn * nS[b];
  } else {
#pragma unroll
    for (int q = 0; q < 5; ++q) qp[q] = plus_value<T, DIM, N>(ft, tb, trc + q * S, code, qm[q]);
  }
  const T gm1 = gamma - 1;
  T irm = 1 / qm[0], irp = 1 / qp[0];
  T um[3] = {qm[1] * irm, qm[2] * irm, qm[3] * irm};
  T up[3] = {qp[1] * irp, qp[2] * irp, qp[3] * irp};
  T rkm = (T)0.5 * (qm[1] * um[0] + qm[2] * um[1] + qm[3] * um[2]);
  T rkp = (T)0.5 * (qp[1] * up[0] + qp[2] * up[1] + qp[3] * up[2]);
  T pm = gm1 * (qm[4] - rkm), pp = gm1 * (qp[4] - rkp);
  T unm = 0, unp = 0;
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    unm += um[comp_of<DIM>(b)] * nS[b];
    unp += up[comp_of<DIM>(b)] * nS[b];
  }
  // lambda |n dS| / 2 with lambda = max(|u-.n|, |u+.n|); the non-stiff
  // terms use it floored at lambda_min |n dS| (lambda_min = 0: unchanged)
  T pen = (T)0.5 * fmax(fabs(unm), fabs(unp));
  const T pns = lambda_min > 0 ? fmax(pen, (T)0.5 * lambda_min * sqrt(n2)) : pen;
  const int64_t nH = ft.nH;
  put<T>(slot, hbuf, S, nH, 0, sm, code, (T)0.5 * (qm[0] * unm + qp[0] * unp) + pns * (qm[0] - qp[0]));
#pragma unroll
  for (int c = 0; c < 3; ++c)
    put<T>(slot, hbuf, S, nH, 1 + c, sm, code,
           (T)0.5 * (qm[1 + c] * unm + qp[1 + c] * unp) + pns * (qm[1 + c] - qp[1 + c]));
  put<T>(slot, hbuf, S, nH, 4, sm, code, (T)0.5 * (rkm * unm + rkp * unp) + pns * (rkm - rkp));
  T pav = (T)0.5 * (pm + pp);
  put<T>(slot, hbuf, S, nH, 5, sm, code, pav * nS[0]);
  put<T>(slot, hbuf, S, nH, 6, sm, code, DIM == 3 ? pav * nS[DIM == 3 ? 1 : 0] : (T)0);
  put<T>(slot, hbuf, S, nH, 7, sm, code, pav * nS[DIM - 1]);
  put<T>(slot, hbuf, S, nH, 8, sm, code,
         (T)0.5 * gamma / gm1 * (pm * unm + pp * unp) + pen * (pm - pp) / gm1);
}

// ---------------------------------------------------------------------------
// cell kernels (one thread per node, EPB cells per block)
// ---------------------------------------------------------------------------
// M multiplies the cells per block (tile size picked by the autotuner).
template <int DIM, int N, int M = 1> struct CellShape {
  static constexpr int NP = ipow(N, DIM);
  static constexpr int EPB = M * (NP >= 256 ? 1 : 256 / NP);
  static constexpr int THREADS = EPB * NP;
  static constexpr int NFP = ipow(N, DIM - 1);
  static constexpr int NF = 2 * DIM;
};

// ---------------------------------------------------------------------------
// nodal change of basis per cell (Gauss-Lobatto <-> Gauss-Legendre nodes):
// out = (B x B [x B]) in for nfld fields (field stride Nn); in == out is
// allowed (a block reads a cell's values before it writes them)
// ---------------------------------------------------------------------------
template <typename T, int DIM, int N>
__global__ void __launch_bounds__(CellShape<DIM, N>::THREADS)
    k_basis(const T* in, T* out, int nfld, int64_t E, Mat1D<T> B) {
  using CS = CellShape<DIM, N>;
  constexpr int NP = CS::NP, EPB = CS::EPB;
  __shared__ T sv[2][EPB][NP];
  __shared__ T sB[N][N];   // the matrix in shared memory (per-thread row index)
  if (threadIdx.x < N * N) sB[threadIdx.x / N][threadIdx.x % N] = B.m[threadIdx.x / N][threadIdx.x % N];
  const int le = threadIdx.x / NP, i = threadIdx.x % NP;
  const int64_t e = (int64_t)blockIdx.x * EPB + le;
  const bool active = e < E;
  const int64_t Nn = E * NP;
  const int64_t node = active ? e * NP + i : 0;
  int idx[3];
  node_index<DIM, N>(i, idx);
  for (int q = 0; q < nfld; ++q) {
    T v = active ? in[q * Nn + node] : (T)0;
    int cur = 0;
    sv[cur][le][i] = v;
    __syncthreads();
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int stride = a == 0 ? 1 : (a == 1 ? N : N * N);
      const int i0 = i - idx[a] * stride;
      T acc = 0;
#pragma unroll
      for (int k = 0; k < N; ++k) acc += sB[idx[a]][k] * sv[cur][le][i0 + k * stride];
      cur ^= 1;
      sv[cur][le][i] = acc;
      v = acc;
      __syncthreads();
    }
    if (active) out[q * Nn + node] = v;
    __syncthreads();
  }
}

// metric terms that vanish on terrain-following cells (x = x(xi_1), y =
// y(xi_2)): reference direction a, physical component b
template <int DIM>
__host__ __device__ constexpr bool kzero(int a, int b) {
  return DIM == 3 ? ((a == 0 && b != 0) || (a == 1 && b != 1)) : (a == 0 && b == 1);
}

// reference directions a with K_ab != 0 (all of them unless terrain-following)
template <int DIM>
__device__ __forceinline__ int amask_of(int terrain, int b) {
  int msk = 0;
#pragma unroll
  for (int a = 0; a < DIM; ++a)
    if (!(terrain && kzero<DIM>(a, b))) msk |= 1 << a;
  return msk;
}

// sum_a sum_k D[k][i_a] * sm[a][line(i, a, k)]  (test-gradient contraction)
// (directions a outside amask are skipped: their fluxes are zero)
template <typename T, int DIM, int N, typename TB>
__device__ __forceinline__ T contract(const TB& tb, const T (*sm)[ipow(N, DIM)], int i,
                                      const int idx[3], int amask = (1 << DIM) - 1) {
  T acc = 0;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    if (!((amask >> a) & 1)) continue;
    const int stride = a == 0 ? 1 : (a == 1 ? N : N * N);
    const int i0 = i - idx[a] * stride;
#pragma unroll
    for (int k = 0; k < N; ++k) acc += tb.D[k][idx[a]] * sm[a][i0 + k * stride];
  }
  return acc;
}

// lift of NFLD slot fields into the residuals of node i
template <typename T, int DIM, int N, int NFLD, typename TB>
__device__ __forceinline__ void lift(const TB& tb, const T* __restrict__ slot, int64_t S,
                                     int64_t e, const int idx[3], T* r) {
  constexpr int NFP = ipow(N, DIM - 1), NF = 2 * DIM;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int a = f >> 1, s = f & 1;
    const T Lv = tb.L[s][idx[a]];
    const int64_t sl = (e * NF + f) * NFP + tang_index<DIM, N>(idx, a);
#pragma unroll
    for (int q = 0; q < NFLD; ++q) r[q] -= __ldg(slot + q * S + sl) * Lv;
  }
}

// Coriolis parameter of a cell: per-cell array if given, else uniform.
__device__ __forceinline__ double coriolis(const double* fcell, double f, int64_t cell) {
  return fcell ? __ldg(fcell + cell) : f;
}

struct PhysK {
  double gamma, g, f;
  const double* fcell = nullptr;   // per-cell Coriolis parameter, or null
  double lambda_min = 0;           // floor of the non-stiff Rusanov coefficient
};

template <typename T, int DIM, int N, int M = 1>
__global__ void __launch_bounds__(CellShape<DIM, N, M>::THREADS)
k_volume_explicit(const T* __restrict__ q, const T* __restrict__ Kg, const T* __restrict__ invMg,
                  const T* __restrict__ slot, int64_t E, int64_t S, Tables<T> tb, PhysK ph,
                  T* __restrict__ fns, T* __restrict__ fs, int terrain) {
  using CS = CellShape<DIM, N, M>;
  constexpr int NP = CS::NP, EPB = CS::EPB;
  __shared__ T sm[EPB][DIM][NP];
  __shared__ SharedTables<T, N> stb;
  stage_tables<T, N>(tb, stb);
  const int le = threadIdx.x / NP, i = threadIdx.x % NP;
  const int64_t e = (int64_t)blockIdx.x * EPB + le;
  const bool active = e < E;
  const int64_t Nn = E * NP;
  const int64_t node = active ? e * NP + i : 0;
  int idx[3];
  node_index<DIM, N>(i, idx);
  T rho = 1, m[3] = {0, 0, 0}, En = 1, K[DIM][DIM], iM = 0;
  if (active) {
    rho = __ldg(q + node);
#pragma unroll
    for (int c = 0; c < 3; ++c) m[c] = __ldg(q + (1 + c) * Nn + node);
    En = __ldg(q + 4 * Nn + node);
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int b = 0; b < DIM; ++b)
        K[a][b] = (terrain && kzero<DIM>(a, b)) ? (T)0 : __ldg(Kg + (a * DIM + b) * Nn + node);
    iM = __ldg(invMg + node);
  } else {
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int b = 0; b < DIM; ++b) K[a][b] = 0;
  }
  const T gm1 = (T)ph.gamma - 1;
  const T ir = 1 / rho;
  const T u[3] = {m[0] * ir, m[1] * ir, m[2] * ir};
  const T rk = (T)0.5 * (m[0] * u[0] + m[1] * u[1] + m[2] * u[2]);
  const T p = gm1 * (En - rk);
  const T hr = (T)ph.gamma / gm1 * p;
  T ut[DIM];   // contravariant velocity times w det J
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    ut[a] = 0;
#pragma unroll
    for (int b = 0; b < DIM; ++b)
      if (!(terrain && kzero<DIM>(a, b))) ut[a] += K[a][b] * u[comp_of<DIM>(b)];
  }
  T r[9];
  // flux fields: 0 rho, 1-3 m_c, 4 rho kappa (advective); 5-7 p e_c, 8 h rho (stiff)
#pragma unroll
  for (int fld = 0; fld < 9; ++fld) {
    const bool skip = (DIM == 2 && fld == 6);   // no y-derivative in the x-z slice
    if (skip) {
      r[fld] = 0;
      continue;
    }
    // pressure fluxes p K_ab e_b: directions with K_ab = 0 drop out
    const int pb = DIM == 3 ? fld - 5 : (fld == 5 ? 0 : 1);
    const int msk = (fld >= 5 && fld <= 7) ? amask_of<DIM>(terrain, pb) : (1 << DIM) - 1;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      if (!((msk >> a) & 1)) continue;
      T v;
      if (fld == 0) v = rho * ut[a];
      else if (fld <= 3) v = m[fld - 1] * ut[a];
      else if (fld == 4) v = rk * ut[a];
      else if (fld <= 7) v = p * K[a][pb];
      else v = hr * ut[a];
      sm[le][a][i] = v;
    }
    __syncthreads();
    r[fld] = contract<T, DIM, N>(stb, sm[le], i, idx, msk);
    __syncthreads();
  }
  if (!active) return;
  lift<T, DIM, N, 9>(stb, slot, S, e, idx, r);
#pragma unroll
  for (int fld = 0; fld < 5; ++fld) fns[fld * Nn + node] = iM * r[fld];
  const T f = (T)coriolis(ph.fcell, ph.f, e), g = (T)ph.g;
  fs[0 * Nn + node] = iM * r[5] + f * m[1];
  fs[1 * Nn + node] = iM * r[6] - f * m[0];
  fs[2 * Nn + node] = iM * r[7] - g * rho;
  fs[3 * Nn + node] = iM * r[8] - g * m[2];
}

// ---------------------------------------------------------------------------
// implicit operator pieces
// ---------------------------------------------------------------------------

// centred weak-gradient flux {x} n dS (DIM fields) and the implicit Rusanov
// jump pc * (x- - x+) (field DIM), pc = a_dt/2 max(|u-.n dS|, |u+.n dS|)
template <typename T, int DIM, int N>
__global__ void k_face_grad(FaceTopo ft, const T* __restrict__ trc, const T* __restrict__ pcoef,
                            T* __restrict__ slot, T* __restrict__ hbuf, Tables<T> tb) {
  int64_t p = ft.p0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= ft.nF) return;
  int sm = __ldg(ft.fp_minus + p), code = __ldg(ft.fp_plus + p);
  T xm = __ldg(trc + sm);
  T xp = plus_value<T, DIM, N>(ft, tb, trc, code, xm);
  T avg = code == -1 ? xm : (T)0.5 * (xm + xp);
#pragma unroll
  for (int b = 0; b < DIM; ++b)
    put<T>(slot, hbuf, ft.S, ft.nH, b, sm, code, -avg * __ldg(geo_ptr<T>(ft) + b * ft.nF + p));
  T pen = (code == -1 || pcoef == nullptr) ? (T)0 : __ldg(pcoef + p) * (xm - xp);
  put<T>(slot, hbuf, ft.S, ft.nH, DIM, sm, code, -pen);
}

// central flux of h rho w:  -{h rho w}.n dS  (zero on walls)
template <typename T, int DIM, int N>
__global__ void k_face_div(FaceTopo ft, const T* __restrict__ trc, const T* __restrict__ trh,
                           T* __restrict__ slot, T* __restrict__ hbuf, Tables<T> tb) {
  int64_t p = ft.p0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= ft.nF) return;
  int sm = __ldg(ft.fp_minus + p), code = __ldg(ft.fp_plus + p);
  T avg = 0;
  if (code != -1) {
    T hm = __ldg(trh + sm), hp = plus_value<T, DIM, N>(ft, tb, trh, code, hm);
    T fm = 0, fp = 0;
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      T n = __ldg(geo_ptr<T>(ft) + b * ft.nF + p);
      T wm = __ldg(trc + b * ft.S + sm);
      T wp = plus_value<T, DIM, N>(ft, tb, trc + b * ft.S, code, wm);
      fm += wm * n;
      fp += wp * n;
    }
    avg = (T)0.5 * (hm * fm + hp * fp);
  }
  put<T>(slot, hbuf, ft.S, ft.nH, 0, sm, code, -avg);
}

// lambda coefficient of the implicit Rusanov term from u_lag traces
template <typename T, int DIM, int N>
__global__ void k_face_lambda(FaceTopo ft, const T* __restrict__ tru, T a_dt_half, T* __restrict__ pcoef,
                              Tables<T> tb) {
  int64_t p = ft.p0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= ft.nF) return;
  int sm = __ldg(ft.fp_minus + p), code = __ldg(ft.fp_plus + p);
  const int g = code == -1 ? far_index(ft, p) : -1;
  const T* fq = far_ptr<T>(ft);
  T unm = 0, unp = 0;
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    T n = __ldg(geo_ptr<T>(ft) + b * ft.nF + p);
    T um = __ldg(tru + comp_of<DIM>(b) * ft.S + sm);
    // far field: the outer state's velocity
    T up = g >= 0 ? __ldg(fq + (1 + comp_of<DIM>(b)) * ft.nFar + g) / __ldg(fq + g)
                  : plus_value<T, DIM, N>(ft, tb, tru + comp_of<DIM>(b) * ft.S, code, um);
    unm += um * n;
    unp += up * n;
  }
  pcoef[p] = a_dt_half * fmax(fabs(unm), fabs(unp));
}

enum GradMode { GRAD_VMULT = 0, GRAD_RECOVER = 1 };

struct ImplK {
  double gamma, g, f, a_dt;
  int r2;
  const double* fcell;   // per-cell Coriolis parameter, or null for the uniform f
  int np;                // nodes per cell (to map a node to its cell)
  // FP32 copies: FP32 kernels must issue no FP64 instruction (GB300 runs
  // FP64 at 1/64 of the FP32 rate, so even a cast per node shows)
  float gamma_f, g_f, adt_f, f_f;
  const float* fcell32;
  // host-folded constants: 1/(1 + beta^2) for a uniform f, (gamma-1) a_dt^2 g
  double dbeta, cgrav;
  float dbeta_f, cgrav_f;
  int penalty;           // implicit Rusanov term on (far-field outer data included)
  // FP32-pair copies (DG_PAIRS kernels): converting a double in the kernel
  // would issue FP64 instructions in every thread
  df64 gamma_p, g_p, adt_p, dbeta_p, cgrav_p, beta_p;
};

// 1/rho of the frozen stage density (read by the gradient cell kernel)
template <typename T>
__global__ void k_recip(const T* __restrict__ a, T* __restrict__ b, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (T)1 / a[i];
}

// kernel parameter in the kernel's precision
template <typename T> __device__ __forceinline__ T kp(double d, float f, df64 p);
template <> __device__ __forceinline__ double kp<double>(double d, float, df64) { return d; }
template <> __device__ __forceinline__ float kp<float>(double, float f, df64) { return f; }
template <> __device__ __forceinline__ df64 kp<df64>(double, float, df64 p) { return p; }

// beta = a_dt f of cell e (Section 3.1)
template <typename T> __device__ __forceinline__ T beta_of(const ImplK& ph, int64_t e);
template <> __device__ __forceinline__ double beta_of<double>(const ImplK& ph, int64_t e) {
  return ph.a_dt * coriolis(ph.fcell, ph.f, e);
}
template <> __device__ __forceinline__ float beta_of<float>(const ImplK& ph, int64_t e) {
  return ph.adt_f * (ph.fcell32 ? __ldg(ph.fcell32 + e) : ph.f_f);
}
template <> __device__ __forceinline__ df64 beta_of<df64>(const ImplK& ph, int64_t e) {
  return ph.fcell ? df64(ph.a_dt * __ldg(ph.fcell + e)) : ph.beta_p;
}

// Per-node metric K_ab = w det(J) (J^{-1})_ab and 1/(w det J) of the
// implicit-operator cell kernels: loaded from stored arrays, or (when `lv`
// is set) recomputed from the cell's corner offsets relative to its first
// corner.  The FP32 engine recomputes: that trades 4 (d^2 + 1) bytes per
// node for about 30 d^2 FP32 flops, which GB300 has in excess.
template <typename T>
struct CellGeo {
  const T* K;
  const T* invM;
  const T* lv;          // n_elem x 2^d x d corner offsets, or null
  const T* tc;          // terrain-following: 16 coefficients per cell, or null
  T x[MAX_N], w[MAX_N]; // Gauss-Legendre nodes and weights on [0, 1]
  int terrain;          // every cell terrain-following: K_ab = 0 where kzero(a, b)
};


// Shared copy of the Gauss-Legendre nodes and weights for the FP32 metric
// recomputation (one thread writes, after the block's first barrier all read).
template <typename T, int N>
__device__ __forceinline__ void stage_nodes(const CellGeo<T>& g, T* sxw) {
  if (std::is_same<T, float>::value && threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      sxw[k] = g.x[k];
      sxw[N + k] = g.w[k];
    }
  }
}

// Cofactors C_ab = det(J) (J^{-1})_ab of the cell map at reference point xi
// and det J, from the cell's corner offsets V relative to its first corner
// (the FP32 recomputation path).  On terrain-following cells only the
// vertical row of J varies (x = x0 + dx xi_1, y = y0 + dy xi_2; dx, dy are
// the offsets of corners 1 and 2), and the entries that vanish exactly are
// set to zero.
template <typename T, int DIM>
__device__ __forceinline__ void corner_cofactors(const T* __restrict__ V, int terrain, const T xi[3],
                                                 T K[DIM][DIM], T& det) {
  if (terrain) {
    T Jz[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) Jz[c] = 0;
#pragma unroll
    for (int v = 1; v < (1 << DIM); ++v) {
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        T wgt = 1;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
          const int bit = (v >> a) & 1;
          if (a == c) wgt *= bit ? (T)1 : (T)-1;
          else wgt *= bit ? xi[a] : (T)1 - xi[a];
        }
        Jz[c] += wgt * __ldg(V + v * DIM + DIM - 1);
      }
    }
    const T dx = __ldg(V + 1 * DIM + 0);
    if (DIM == 2) {
      K[0][0] = Jz[1];
      K[0][1] = 0;
      K[1][0] = -Jz[0];
      K[1][1] = dx;
      det = dx * Jz[1];
    } else {
      const T dy = __ldg(V + 2 * DIM + 1);
      K[0][0] = dy * Jz[2];
      K[1][1] = Jz[2] * dx;
      K[2][0] = -(Jz[0] * dy);
      K[2][1] = -(dx * Jz[1]);
      K[2][2] = dx * dy;
      K[0][1] = K[0][2] = K[1][0] = K[1][2] = 0;
      det = dx * K[0][0];
    }
    return;
  }
  T J[DIM][DIM];   // J[b][c] = d x_b / d xi_c
#pragma unroll
  for (int b = 0; b < DIM; ++b)
#pragma unroll
    for (int c = 0; c < DIM; ++c) J[b][c] = 0;
#pragma unroll
  for (int v = 1; v < (1 << DIM); ++v) {   // corner 0 is the origin
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      T wgt = 1;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const int bit = (v >> a) & 1;
        if (a == c) wgt *= bit ? (T)1 : (T)-1;
        else wgt *= bit ? xi[a] : (T)1 - xi[a];
      }
#pragma unroll
      for (int b = 0; b < DIM; ++b) J[b][c] += wgt * __ldg(V + v * DIM + b);
    }
  }
  if (DIM == 2) {
    K[0][0] = J[1][1];
    K[0][1] = -J[0][1];
    K[1][0] = -J[1][0];
    K[1][1] = J[0][0];
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  } else {
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int c1 = (a + 1) % 3, c2 = (a + 2) % 3;
      K[a][0] = J[1][c1] * J[2][c2] - J[2][c1] * J[1][c2];
      K[a][1] = J[2][c1] * J[0][c2] - J[0][c1] * J[2][c2];
      K[a][2] = J[0][c1] * J[1][c2] - J[1][c1] * J[0][c2];
    }
    det = J[0][0] * K[0][0] + J[1][0] * K[0][1] + J[2][0] * K[0][2];
  }
}

// Cofactors and det J of a terrain-following cell at xi from its 16
// coefficients t (dx, dy, then bilinear coefficients of the vertical row of
// J): the same formulas as the terrain branch of corner_cofactors with the
// corner sums folded per cell.
template <typename T, int DIM>
__device__ __forceinline__ void terrain_row(const T* t, const T xi[3], T K[DIM][DIM], T& det) {
  const T Jz0 = (t[2] + t[3] * xi[1]) + xi[2] * (t[4] + t[5] * xi[1]);
  const T Jz1 = (t[6] + t[7] * xi[0]) + xi[2] * (t[8] + t[9] * xi[0]);
  const T dx = t[0];
  if (DIM == 2) {
    K[0][0] = Jz1;
    K[0][1] = 0;
    K[1][0] = -Jz0;
    K[1][1] = dx;
    det = dx * Jz1;
  } else {
    const T Jz2 = (t[10] + t[11] * xi[0]) + xi[1] * (t[12] + t[13] * xi[0]);
    const T dy = t[1];
    K[0][0] = dy * Jz2;
    K[1][1] = Jz2 * dx;
    K[2][0] = -(Jz0 * dy);
    K[2][1] = -(dx * Jz1);
    K[2][2] = dx * dy;
    K[0][1] = K[0][2] = K[1][0] = K[1][2] = 0;
    det = dx * K[0][0];
  }
}

// tcs: the cell's terrain coefficients (shared memory), FP32 only
template <typename T, int DIM, int N>
__device__ __forceinline__ void node_metric(const CellGeo<T>& g, int64_t e, int64_t node, int64_t Nn,
                                            const int idx[3], T K[DIM][DIM], T& iM, const T* sxw = nullptr,
                                            const T* tcs = nullptr) {
  // FP64 always loads the stored metric (the FP64 geometry has no corner
  // offsets); only FP32 recomputes it
  if (!std::is_same<T, float>::value || g.lv == nullptr) {
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int b = 0; b < DIM; ++b)
        K[a][b] = (g.terrain && kzero<DIM>(a, b)) ? (T)0 : __ldg(g.K + (a * DIM + b) * Nn + node);
    iM = __ldg(g.invM + node);
    return;
  }
  T xi[3] = {0, 0, 0}, wq = 1;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    // nodes and weights from the block's shared copy (sxw[0..N), sxw[N..2N)):
    // indexing the parameter arrays per thread would copy them to local memory
    xi[a] = sxw[idx[a]];
    wq *= sxw[N + idx[a]];
  }
  T det;
  if (tcs)
    terrain_row<T, DIM>(tcs, xi, K, det);
  else
    corner_cofactors<T, DIM>(g.lv + e * (DIM << DIM), g.terrain, xi, K, det);
#pragma unroll
  for (int a = 0; a < DIM; ++a)
#pragma unroll
    for (int b = 0; b < DIM; ++b) K[a][b] *= wq;
  iM = 1 / (wq * det);
}

enum DivMode { DIV_VMULT = 0, DIV_RHS = 1 };

// u* = rho^{-1} (I + beta J)^{-1} (m_hat - a_dt g rho k)           (R2)
// u* = rho^{-1} (m_hat - a_dt f rho k x u_lag - a_dt g rho k)       (R1)
template <typename T>
__global__ void k_ustar(const T* __restrict__ mhat, const T* __restrict__ rho, const T* __restrict__ ulag,
                        int64_t Nn, ImplK ph, T* __restrict__ ustar) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= Nn) return;
  const T rh = rho[k], adt = (T)ph.a_dt;
  T v0 = mhat[k], v1 = mhat[Nn + k], v2 = mhat[2 * Nn + k] - adt * (T)ph.g * rh;
  const T ir = 1 / rh;
  const double fc = coriolis(ph.fcell, ph.f, k / ph.np);
  if (ph.r2) {
    const T beta = (T)(ph.a_dt * fc), d = 1 / (1 + beta * beta);
    ustar[k] = (v0 + beta * v1) * d * ir;
    ustar[Nn + k] = (v1 - beta * v0) * d * ir;
    ustar[2 * Nn + k] = v2 * ir;
  } else {
    const T fr = adt * (T)fc * rh;
    // k x u = (-v, u, 0)
    ustar[k] = (v0 + fr * ulag[Nn + k]) * ir;
    ustar[Nn + k] = (v1 - fr * ulag[k]) * ir;
    ustar[2 * Nn + k] = v2 * ir;
  }
}

}  // namespace dg
