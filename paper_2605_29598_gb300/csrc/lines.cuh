// Line-per-thread form of the two fused Schur-vmult passes (3D, n = 4 nodes
// per direction, degree 3): the same operators as k_grad_fused /
// k_div_fused in VMULT mode (Section 3: the weak gradient with centred face
// values and the implicit Rusanov jump, then the weak divergence of h rho w
// with the centred face flux), with fewer issued instructions per node.
//
// A cell is served by n^2 = 16 threads; thread t = jy + n jz owns the x-line
// of nodes (0..n-1, jy, jz), which is 16 contiguous bytes (FP32) in the
// element-major layout, so its values, the coefficients on it and the
// results move with 128-bit loads and stores.  On that line:
//  - the x-direction contraction and both x-faces' traces and lifts stay in
//    registers with compile-time table entries;
//  - the y and z contractions read the staged flux components of the whole
//    cell with one 128-bit shared load per quadrature point (the four
//    values along x share the table entry of the thread's own jy or jz);
//  - the thread evaluates one point of every face: (jy, jz) on the x-faces,
//    (x = jy, z = jz) on the y-faces, (x = jy, y = jz) on the z-faces, so the
//    face work is spread evenly; the lift values of the y and z faces pass
//    through shared memory and are read back 128 bits at a time.
// Staged cells use a padded z-plane stride (n^2 + 4 values) so that the
// strided y- and z-line reads of the face traces are free of bank conflicts.
// The gradient pass fetches the neighbours' lines with asynchronous copies
// into shared memory as soon as the face codes arrive and reads them only
// after its own volume work, so the second of its two dependent global
// round trips is hidden (the kernels are bound by load latency, not by
// bandwidth or issue).  Having w, it also writes g = (h rho)- (w- . n dS)
// at every own face point; the divergence pass then forms each face flux
// from its own g and the neighbour's, two values per face point instead of
// three neighbour lines, the own traces and the normals.
// The kernels serve terrain-following meshes (five metric terms per node;
// every mesh of the paper's workloads); the host keeps the other schedules
// for general cells.
#pragma once

#include "fused.cuh"

namespace dg {

template <int EPB_>
struct LineShape {
  static constexpr int N = 4, NP = 64, NFP = 16, NF = 6, NSL = NF * NFP;
  static constexpr int EPB = EPB_;
  static constexpr int PL = N * N + 4;   // padded z-plane stride of a staged cell
  static constexpr int CSZ = N * PL;     // staged cell
  // staged flux components, read as 128-bit rows only (conflict-free
  // without padding)
  static constexpr int FPL = N * N, FSZ = N * FPL;
  static constexpr int THREADS = EPB * NFP;
};

// 4 consecutive values, 16-byte aligned: global read-only loads, global
// stores, shared loads and shared stores
template <typename T> __device__ __forceinline__ void ld4g(const T* __restrict__ p, T v[4]);
template <> __device__ __forceinline__ void ld4g<float>(const float* __restrict__ p, float v[4]) {
  const float4 q = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
template <> __device__ __forceinline__ void ld4g<double>(const double* __restrict__ p, double v[4]) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
template <> __device__ __forceinline__ void ld4g<df64>(const df64* __restrict__ p, df64 v[4]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  v[0] = df64(a.x, a.y); v[1] = df64(a.z, a.w); v[2] = df64(b.x, b.y); v[3] = df64(b.z, b.w);
}
template <typename T> __device__ __forceinline__ void st4(T* p, const T v[4]);
template <> __device__ __forceinline__ void st4<float>(float* p, const float v[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <> __device__ __forceinline__ void st4<double>(double* p, const double v[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
template <> __device__ __forceinline__ void st4<df64>(df64* p, const df64 v[4]) {
  reinterpret_cast<float4*>(p)[0] = make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo);
  reinterpret_cast<float4*>(p)[1] = make_float4(v[2].hi, v[2].lo, v[3].hi, v[3].lo);
}
template <typename T> __device__ __forceinline__ void ld4s(const T* p, T v[4]);
template <> __device__ __forceinline__ void ld4s<float>(const float* p, float v[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
template <> __device__ __forceinline__ void ld4s<double>(const double* p, double v[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
template <> __device__ __forceinline__ void ld4s<df64>(const df64* p, df64 v[4]) {
  const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
  v[0] = df64(a.x, a.y); v[1] = df64(a.z, a.w); v[2] = df64(b.x, b.y); v[3] = df64(b.z, b.w);
}

// Terrain-following cells only (every cell x = x(xi_1), y = y(xi_2)): of
// the metric K_ab = w det(J) (J^{-1})_ab the five terms that do not vanish,
// in the order K00, K11, K20, K21, K22 (stored-array index a * 3 + b below),
// and 1/(w det J), on the thread's own x-line nodes (ix, jy, jz).  FP64 and
// pairs load the stored metric; FP32 recomputes it from the cell's 16
// terrain coefficients (tcs, shared).  xj, xk: the nodes at jy and jz; wjk:
// the product of their weights.  Indices are 32-bit: the host takes this
// schedule only while every offset fits.
__host__ __device__ constexpr int line_term(int j) { return j == 0 ? 0 : (j == 1 ? 4 : j + 4); }

template <typename T>
__device__ __forceinline__ void line_metric(const CellGeo<T>& g, int n0, int Nn, T xj, T xk, T wjk,
                                            const T* tcs, T Kt[5][4], T iM[4]) {
  if constexpr (std::is_same<T, float>::value) {
    if (tcs) {
#pragma unroll
      for (int ix = 0; ix < 4; ++ix) {
        const float xi[3] = {g.x[ix], xj, xk};
        const float wq = g.w[ix] * wjk;
        float K[3][3], det;
        terrain_row<float, 3>(tcs, xi, K, det);
        Kt[0][ix] = K[0][0] * wq;
        Kt[1][ix] = K[1][1] * wq;
        Kt[2][ix] = K[2][0] * wq;
        Kt[3][ix] = K[2][1] * wq;
        Kt[4][ix] = K[2][2] * wq;
        iM[ix] = __frcp_rn(wq * det);
      }
      return;
    }
  }
#pragma unroll
  for (int j = 0; j < 5; ++j) ld4g<T>(g.K + (int64_t)line_term(j) * Nn + n0, Kt[j]);
  ld4g<T>(g.invM + n0, iM);
}

// Outward n dS at the thread's point of face f (tangential nodes xj, xk in
// increasing direction order): loaded per slot (FP64, pairs) or recomputed
// from the terrain coefficients (FP32), as slot_normal does.
template <typename T>
__device__ __forceinline__ void line_face_normal(const T* __restrict__ snS, int S, int f, int sl, T xj, T xk,
                                                 T wjk, const T* tcs, T nS[3]) {
  if (!std::is_same<T, float>::value || snS) {
#pragma unroll
    for (int b = 0; b < 3; ++b) nS[b] = __ldg(snS + b * S + sl);
    return;
  }
  const int a = f >> 1, s = f & 1;
  T xi[3];
  xi[a] = (T)s;
  xi[a == 0 ? 1 : 0] = xj;
  xi[a == 2 ? 1 : 2] = xk;
  T C[3][3], det;
  terrain_row<T, 3>(tcs, xi, C, det);
  const T sw = s ? wjk : -wjk;
#pragma unroll
  for (int b = 0; b < 3; ++b) nS[b] = sw * C[a][b];
}

// Asynchronous global -> shared copies (cp.async): the neighbours' lines
// are in flight while the thread does the cell's own volume work, and are
// waited for (cp.async.wait_all, each thread its own copies) only before
// the face fluxes.  16-byte copies need 16-byte aligned addresses on both
// sides; smaller ones the element's alignment.
template <int B>
__device__ __forceinline__ void cp_async(void* s, const void* g) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(s));
  if constexpr (B == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(g), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// the neighbour's line through the thread's point of face f, copied raw to
// dst (4 values, 16-byte aligned): x-lines in 16-byte pieces, y- and
// z-lines value by value
template <typename T>
__device__ __forceinline__ void plus_line_async(const T* __restrict__ nb, int f, int t, int jy, int jz, T* dst) {
  const int a = f >> 1;
  if (a == 0) {
#pragma unroll
    for (int h = 0; h < (int)(4 * sizeof(T) / 16); ++h)
      cp_async<16>(reinterpret_cast<char*>(dst) + 16 * h, reinterpret_cast<const char*>(nb + 4 * t) + 16 * h);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      cp_async<(int)sizeof(T)>(dst + k, nb + (a == 1 ? jy + 4 * k + 16 * jz : jy + 4 * jz + 16 * k));
  }
}

// the copied line contracted to the neighbour's face f ^ 1
template <typename T>
__device__ __forceinline__ T plus_from(const Tables<T>& tb, const T* v, int f) {
  const int s = (f & 1) ^ 1;
  T acc = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) acc += tb.L[s][k] * v[k];
  return acc;
}

// Butterfly exchange of one value with lane ^ m (pairs: both halves).
__device__ __forceinline__ float shfl_x(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ double shfl_x(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ df64 shfl_x(df64 v, int m) {
  return df64(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}

// Reduce-scatter over the four lanes whose lane numbers differ in the two
// bits of unit m (m = 1: the lanes of one jz, q = jy; m = 4: the lanes of
// one jy, q = jz): the lane at position q of its group returns the group's
// sum of v[q].  Three exchanges; every lane of the warp must take part.
template <typename T>
__device__ __forceinline__ T reduce_scatter4(const T v[4], int q, int m) {
  const bool h = (q >> 1) & 1, l = q & 1;
  const T a0 = (h ? v[2] : v[0]) + shfl_x(h ? v[0] : v[2], 2 * m);
  const T a1 = (h ? v[3] : v[1]) + shfl_x(h ? v[1] : v[3], 2 * m);
  return (l ? a1 : a0) + shfl_x(l ? a0 : a1, m);
}

// own trace at the thread's point of face f from the staged cell (stride PL
// between z-planes) or, on x-faces, from the thread's registers
template <typename T, int PL>
__device__ __forceinline__ T own_trace(const Tables<T>& tb, const T* sc, const T xl[4], int f, int jy, int jz) {
  const int a = f >> 1, s = f & 1;
  T acc = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const T v = a == 0 ? xl[k] : sc[a == 1 ? jy + 4 * k + PL * jz : jy + 4 * jz + PL * k];
    acc += tb.L[s][k] * v;
  }
  return acc;
}

// cells per block for the tile multiplier M (1, 2, 4); 8-byte types stop at
// 4 cells (static shared memory stays below 48 KB)
template <typename T>
constexpr int line_epb(int M) {
  return sizeof(T) == 4 ? 2 * M : (M >= 2 ? 4 : 2);
}

// resident blocks per SM asked of the register allocator: FP32 at most
// REG32 registers per thread (more resident warps hide the load latency
// that binds these kernels; 80 in the gradient pass, 72 in the lighter
// divergence pass, the most each fits without spilling), the 8-byte types
// up to 255
constexpr int kLineReg32 = 80;
template <typename T, int EPB, int REG32 = kLineReg32>
struct LineOcc {
  static constexpr int MIN_BLOCKS = sizeof(T) == 4 ? 65536 / (REG32 * EPB * 16) : 256 / (EPB * 16);
};
constexpr int kLineReg32Div = 72;

// Gradient pass (VMULT): w = rho^{-1} (I + beta J)^{-1} G (R2) or G / rho
// (R1); y = x + pen - (gamma-1) a_dt^2 g G_z (R2).  Same arguments and
// face semantics as k_grad_fused (cell face codes: >= 0 neighbour, -1
// wall, -2 2:1 face with slot values, -3 far field).
template <typename T, int EPB>
__global__ void __launch_bounds__(LineShape<EPB>::THREADS, LineOcc<T, EPB>::MIN_BLOCKS)
k_grad_lines(const T* __restrict__ x, const int* __restrict__ cface, const T* __restrict__ snS,
             const T* __restrict__ pcs, const T* __restrict__ irho, CellGeo<T> geo, const T* __restrict__ slot,
             int E, int S, Tables<T> tb, ImplK ph, T* __restrict__ wv, T* __restrict__ y,
             const T* __restrict__ trh, T* __restrict__ gout) {
  using LS = LineShape<EPB>;
  constexpr int N = LS::N, NP = LS::NP, NFP = LS::NFP, NF = LS::NF, NSL = LS::NSL, PL = LS::PL, CSZ = LS::CSZ;
  constexpr int FPL = LS::FPL, FSZ = LS::FSZ;
  __shared__ __align__(16) T sx[EPB][CSZ];
  // -x K_ab staged for the y and z contractions: (a, b) = (2, 0), (1, 1), (2, 1), (2, 2)
  __shared__ __align__(16) T sF[EPB][4][FSZ];
  __shared__ __align__(16) T slf[EPB][4][4][NFP];   // lift values of faces 2..5, fields 0..3
  // per face: the penalty coefficient and the neighbour's line through the
  // thread's point, each thread's own (asynchronous copies)
  __shared__ T spen[EPB][NF][NFP];
  __shared__ __align__(16) T snb[EPB][NF][NFP][4];
  __shared__ T shm[EPB][NF][NFP];                   // own h rho traces (for gout)
  __shared__ __align__(16) T stc[std::is_same<T, float>::value ? EPB : 1][16];
  __shared__ SharedTables<T, N> stb;
  __shared__ T sxw[2 * N];
  const int c = threadIdx.x / NFP, t = threadIdx.x % NFP, jy = t % N, jz = t / N;
  const int e0 = blockIdx.x * EPB, e = e0 + c;
  const bool active = e < E;
  const int Nn = E * NP;
  const int n0 = (active ? e : 0) * NP + N * t;
  const bool tcell = std::is_same<T, float>::value && geo.tc != nullptr;
  stage_terrain<T, EPB>(geo, e0, E, stc);
  stage_tables<T, N>(tb, stb);
  stage_nodes_all<T, N>(geo, sxw);
  T xl[N] = {0, 0, 0, 0};
  if (active) ld4g<T>(x + n0, xl);
  st4<T>(&sx[c][N * jy + PL * jz], xl);
  // global reads first: face codes, then the neighbours' lines and the
  // penalties as asynchronous copies, 1/rho
  int codes[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int code = active ? __ldg(cface + e * NF + f) : -1;
    codes[f] = code;
    const int sl = e * NSL + f * NFP + t;
    if (code >= 0) plus_line_async<T>(x + code * NP, f, t, jy, jz, snb[c][f][t]);
    if ((code >= 0 || code == -3) && pcs)
      cp_async<(int)sizeof(T)>(&spen[c][f][t], pcs + sl);
    else
      spen[c][f][t] = 0;
    if (code >= 0 || code == -3)
      cp_async<(int)sizeof(T)>(&shm[c][f][t], trh + sl);
    else
      shm[c][f][t] = 0;
  }
  T ir[N] = {0, 0, 0, 0};
  if (active) ld4g<T>(irho + n0, ir);
  __syncthreads();
  const T xj = sxw[jy], xk = sxw[jz], wjk = sxw[N + jy] * sxw[N + jz];
  const T* tcs = tcell ? stc[c] : nullptr;
  // volume term: the x-direction in registers, the others staged
  T r[4][N], iM[N];
  {
    T Kt[5][N];
    line_metric<T>(geo, n0, Nn, xj, xk, wjk, tcs, Kt, iM);
    T F[N];
#pragma unroll
    for (int k = 0; k < N; ++k) F[k] = -xl[k] * Kt[0][k];
#pragma unroll
    for (int ix = 0; ix < N; ++ix) {
      r[0][ix] = 0;
#pragma unroll
      for (int k = 0; k < N; ++k) r[0][ix] += tb.D[k][ix] * F[k];
      r[1][ix] = r[2][ix] = r[3][ix] = 0;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
#pragma unroll
      for (int k = 0; k < N; ++k) F[k] = -xl[k] * Kt[j == 0 ? 2 : (j == 1 ? 1 : j + 1)][k];
      st4<T>(&sF[c][j][N * jy + FPL * jz], F);
    }
  }
  // the thread's point of every face (its copies have landed)
  cp_async_wait_all();
  T lx[2][4];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int a = f >> 1, s = f & 1;
    const int code = codes[f];
    const int sl = e * NSL + f * NFP + t;
    T lv[4] = {0, 0, 0, 0};
    if (active) {
      if (code == -2) {
#pragma unroll
        for (int q = 0; q < 4; ++q) lv[q] = __ldg(slot + q * S + sl);
      } else {
        const T xm = own_trace<T, PL>(tb, sx[c], xl, f, jy, jz);
        // wall: {x} = x-, no jump; far field: the linear part (outer value 0)
        const T xpv = code == -1 ? xm : (code >= 0 ? plus_from<T>(tb, snb[c][f][t], f) : (T)0);
        const T avg = code == -1 ? xm : (T)0.5 * (xm + xpv);
        T nS[3];
        line_face_normal<T>(snS, S, f, sl, xj, xk, wjk, tcs, nS);
#pragma unroll
        for (int b = 0; b < 3; ++b) lv[b] = -avg * nS[b];
        lv[3] = code == -1 ? (T)0 : -spen[c][f][t] * (xm - xpv);
      }
    }
    if (a == 0) {
#pragma unroll
      for (int q = 0; q < 4; ++q) lx[s][q] = lv[q];
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) slf[c][f - 2][q][t] = lv[q];
    }
  }
  __syncthreads();
  // y contraction of -x K11 (b = 1), z contractions of -x K2b (b = 0, 1, 2)
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const T dy = stb.D[k][jy], dz = stb.D[k][jz];
    T v1[N], v0[N], v2[N], v3[N];
    ld4s<T>(&sF[c][1][N * k + FPL * jz], v1);
    ld4s<T>(&sF[c][0][N * jy + FPL * k], v0);
    ld4s<T>(&sF[c][2][N * jy + FPL * k], v2);
    ld4s<T>(&sF[c][3][N * jy + FPL * k], v3);
#pragma unroll
    for (int ix = 0; ix < N; ++ix) {
      r[0][ix] += dz * v0[ix];
      r[1][ix] += dy * v1[ix] + dz * v2[ix];
      r[2][ix] += dz * v3[ix];
    }
  }
  // lifts: x-faces from registers, y- and z-faces from the shared values
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const T Ly = stb.L[s][jy], Lz = stb.L[s][jz];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      T vy[N], vz[N];
      ld4s<T>(&slf[c][s][q][N * jz], vy);
      ld4s<T>(&slf[c][2 + s][q][N * jy], vz);
#pragma unroll
      for (int ix = 0; ix < N; ++ix) r[q][ix] -= lx[s][q] * tb.L[s][ix] + vy[ix] * Ly + vz[ix] * Lz;
    }
  }
  T beta = 0, d = 1;
  if (ph.r2) {
    beta = beta_of<T>(ph, active ? e : 0);
    d = (ph.fcell || ph.fcell32) ? (T)1 / (1 + beta * beta) : kp<T>(ph.dbeta, ph.dbeta_f, ph.dbeta_p);
  }
  const T cg = kp<T>(ph.cgrav, ph.cgrav_f, ph.cgrav_p);
  T wo[3][N], yo[N];
#pragma unroll
  for (int ix = 0; ix < N; ++ix) {
    const T G0 = iM[ix] * r[0][ix], G1 = iM[ix] * r[1][ix], G2 = iM[ix] * r[2][ix];
    if (ph.r2) {
      wo[0][ix] = (G0 + beta * G1) * d * ir[ix];
      wo[1][ix] = (G1 - beta * G0) * d * ir[ix];
    } else {
      wo[0][ix] = G0 * ir[ix];
      wo[1][ix] = G1 * ir[ix];
    }
    wo[2][ix] = G2 * ir[ix];
    yo[ix] = xl[ix] + iM[ix] * r[3][ix];
    if (ph.r2) yo[ix] -= cg * G2;
    if (!active) wo[0][ix] = wo[1][ix] = wo[2][ix] = 0;
  }
  if (active) {
#pragma unroll
    for (int b = 0; b < 3; ++b) st4<T>(wv + b * Nn + n0, wo[b]);
    st4<T>(y + n0, yo);
  }
  // For the divergence pass: g = (h rho)- (w- . n dS) at the face points of
  // every conforming, periodic and far-field face (the other side's normal
  // is the negative, so the divergence face flux is -(g_own - g_nb) / 2).
  // The traces of w: x-faces from the thread's line; y- and z-faces summed
  // across the four lanes that hold the line's other nodes, which leaves
  // lane (jy, jz) the y-face point (x = jy, z = jz) and the z-face point
  // (x = jz, y = jy).  Recomputed terrain normals of x- and y-faces have
  // one non-zero component (the others are exact zeros), so one trace of w
  // suffices there.  All lanes run the exchanges (inactive cells with w = 0).
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int a = f >> 1, s = f & 1;
    const T Lq = a == 1 ? stb.L[s][jy] : stb.L[s][jz];
    T tr[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      tr[b] = 0;
      if (tcs && a != 2 && a != b) continue;
      if (a == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) tr[b] += tb.L[s][k] * wo[b][k];
      } else {
        T v[N];
#pragma unroll
        for (int ix = 0; ix < N; ++ix) v[ix] = Lq * wo[b][ix];
        tr[b] = a == 1 ? reduce_scatter4<T>(v, jy, 1) : reduce_scatter4<T>(v, jz, 4);
      }
    }
    // this lane's point of face f and its tangential nodes
    const int p = a == 2 ? jz + N * jy : t;
    const int code = codes[f];   // (the same in every thread of the cell)
    if (!active || (code < 0 && code != -3)) continue;
    const int sl = e * NSL + f * NFP + p;
    T nS[3];
    if (a == 2)
      line_face_normal<T>(snS, S, f, sl, sxw[jz], sxw[jy], wjk, tcs, nS);
    else
      line_face_normal<T>(snS, S, f, sl, xj, xk, wjk, tcs, nS);
    T fm = 0;
#pragma unroll
    for (int b = 0; b < 3; ++b)
      if (!tcs || a == 2 || a == b) fm += tr[b] * nS[b];
    gout[sl] = shm[c][f][p] * fm;
  }
}

// Divergence pass (VMULT): y -= (gamma-1) a_dt^2 Div, Div = M^{-1}[-int h
// rho w . grad(psi) + {h rho w}.n dS (zero on walls)], h rho = gamma p_lag /
// (gamma - 1); the central face flux from the per-slot g = (h rho)- (w- .
// n dS) that the gradient pass writes, this side's and the neighbour's.
template <typename T, int EPB>
__global__ void __launch_bounds__(LineShape<EPB>::THREADS, LineOcc<T, EPB, kLineReg32Div>::MIN_BLOCKS)
k_div_lines(Fields<T> wv, const T* __restrict__ gin, const int* __restrict__ cface, const T* __restrict__ plag,
            CellGeo<T> geo, const T* __restrict__ slot, int E, Tables<T> tb, ImplK ph, T* __restrict__ y) {
  using LS = LineShape<EPB>;
  constexpr int N = LS::N, NP = LS::NP, NFP = LS::NFP, NF = LS::NF, NSL = LS::NSL, FPL = LS::FPL, FSZ = LS::FSZ;
  __shared__ __align__(16) T sF[EPB][2][FSZ];    // -h rho (K w)_a of directions a = 1, 2
  __shared__ __align__(16) T slf[EPB][4][NFP];   // lift values of faces 2..5
  // per face point: g = (h rho w . n dS) of this side and of the neighbour,
  // written by the gradient pass (asynchronous copies, each thread its own)
  __shared__ T sg[EPB][NF][2][NFP];
  __shared__ __align__(16) T stc[std::is_same<T, float>::value ? EPB : 1][16];
  __shared__ SharedTables<T, N> stb;
  __shared__ T sxw[2 * N];
  const int c = threadIdx.x / NFP, t = threadIdx.x % NFP, jy = t % N, jz = t / N;
  const int e0 = blockIdx.x * EPB, e = e0 + c;
  const bool active = e < E;
  const int Nn = E * NP;
  const int n0 = (active ? e : 0) * NP + N * t;
  const bool tcell = std::is_same<T, float>::value && geo.tc != nullptr;
  stage_terrain<T, EPB>(geo, e0, E, stc);
  stage_tables<T, N>(tb, stb);
  stage_nodes_all<T, N>(geo, sxw);
  int codes[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int code = active ? __ldg(cface + e * NF + f) : -1;
    codes[f] = code;
    const int sl = e * NSL + f * NFP + t;
    if (code >= 0 || code == -3)
      cp_async<(int)sizeof(T)>(&sg[c][f][0][t], gin + sl);
    else
      sg[c][f][0][t] = 0;
    if (code >= 0)
      cp_async<(int)sizeof(T)>(&sg[c][f][1][t], gin + (code * NF + (f ^ 1)) * NFP + t);
    else
      sg[c][f][1][t] = 0;
  }
  T wl[3][N];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
#pragma unroll
    for (int ix = 0; ix < N; ++ix) wl[b][ix] = 0;
    if (active) ld4g<T>(wv.f[b] + n0, wl[b]);
  }
  T pl[N] = {0, 0, 0, 0}, yl[N] = {0, 0, 0, 0};
  if (active) {
    ld4g<T>(plag + n0, pl);
    ld4g<T>(y + n0, yl);
  }
  __syncthreads();
  const T xj = sxw[jy], xk = sxw[jz], wjk = sxw[N + jy] * sxw[N + jz];
  const T* tcs = tcell ? stc[c] : nullptr;
  const T gam = kp<T>(ph.gamma, ph.gamma_f, ph.gamma_p);
  const T gm1 = gam - 1;
  const T hcoef = gam / gm1;
  T r[N], iM[N];
  {
    T Kt[5][N];
    line_metric<T>(geo, n0, Nn, xj, xk, wjk, tcs, Kt, iM);
    T F0[N], F1[N], F2[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const T hr = hcoef * pl[k];
      F0[k] = -hr * (Kt[0][k] * wl[0][k]);
      F1[k] = -hr * (Kt[1][k] * wl[1][k]);
      F2[k] = -hr * (Kt[2][k] * wl[0][k] + Kt[3][k] * wl[1][k] + Kt[4][k] * wl[2][k]);
    }
#pragma unroll
    for (int ix = 0; ix < N; ++ix) {
      r[ix] = 0;
#pragma unroll
      for (int k = 0; k < N; ++k) r[ix] += tb.D[k][ix] * F0[k];
    }
    st4<T>(&sF[c][0][N * jy + FPL * jz], F1);
    st4<T>(&sF[c][1][N * jy + FPL * jz], F2);
  }
  // face fluxes -{h rho w}.n dS = -(g_own - g_neighbour) / 2 (the two sides'
  // normals are negatives of each other); far field: the linear part
  // -g_own / 2; wall: the mirror velocity makes the flux vanish; 2:1 faces:
  // the slot values of the face kernels
  cp_async_wait_all();
  T lx[2];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int a = f >> 1, s = f & 1;
    const int code = codes[f];
    const int sl = e * NSL + f * NFP + t;
    T lv = 0;
    if (active && code != -1)
      lv = code == -2 ? __ldg(slot + sl) : -(T)0.5 * (sg[c][f][0][t] - sg[c][f][1][t]);
    if (a == 0)
      lx[s] = lv;
    else
      slf[c][f - 2][t] = lv;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const T dy = stb.D[k][jy], dz = stb.D[k][jz];
    T vy[N], vz[N];
    ld4s<T>(&sF[c][0][N * k + FPL * jz], vy);
    ld4s<T>(&sF[c][1][N * jy + FPL * k], vz);
#pragma unroll
    for (int ix = 0; ix < N; ++ix) r[ix] += dy * vy[ix] + dz * vz[ix];
  }
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const T Ly = stb.L[s][jy], Lz = stb.L[s][jz];
    T vy[N], vz[N];
    ld4s<T>(&slf[c][s][N * jz], vy);
    ld4s<T>(&slf[c][2 + s][N * jy], vz);
#pragma unroll
    for (int ix = 0; ix < N; ++ix) r[ix] -= lx[s] * tb.L[s][ix] + vy[ix] * Ly + vz[ix] * Lz;
  }
  if (!active) return;
  const T adt = kp<T>(ph.a_dt, ph.adt_f, ph.adt_p);
  const T cdiv = gm1 * adt * adt;
#pragma unroll
  for (int ix = 0; ix < N; ++ix) yl[ix] -= cdiv * (iM[ix] * r[ix]);
  st4<T>(y + n0, yl);
}

}  // namespace dg
