// Pieces of the Krylov solver and the ARK2 step shared by the host-driven
// step (solver.cu) and the device-driven step captured as a CUDA graph
// (graph.cu).
#pragma once

#include <cmath>

#include "engine.cuh"

namespace dg {

constexpr int RED_BLOCKS = 608;    // partial sums per reduction (fixed order): 4 blocks per SM
constexpr int MAX_RESTART = 64;

struct Coefs {
  double c[MAX_RESTART + 1];
};

// stage coefficients of k_stage_predict / k_final_update
struct StageCoefs {
  const double* fns[3];
  const double* fs[3];
  double a[3], at[3];
  int nst;
  double dt;
};

struct Red {
  double* partial;   // RED_BLOCKS * (MAX_RESTART + 1)
  double* out;       // MAX_RESTART + 1
};

// generic vmult closure: the solver is written against y = S x
struct Vmult {
  int (*fn)(void* self, const double* x, double* y, cudaStream_t st);
  void* self;
  int operator()(const double* x, double* y, cudaStream_t st) const { return fn(self, x, y, st); }
};

struct SchurCtx {
  dg_mesh* m;
  ImplK k;
  const double* rho;
  const double* plag;
  int penalty;
};

struct Schur32Ctx {
  dg_mesh* m;
  ImplK k;
  const float* rho;
  const float* plag;
  int penalty;
  float* x32;
  float* y32;
};

// DG_PAIRS: the vmult in FP32 pairs behind an FP64 interface
struct SchurDfCtx {
  dg_mesh* m;
  ImplK k;
  const df64* rho;
  const df64* plag;
  int penalty;
  df64* xdf;
  df64* ydf;
};

// ARK2 (TR-BDF2) tableaux of Section 3: explicit a, implicit at, weights b
struct Ark2 {
  double a[3][3], at[3][3], b[3];
  Ark2() {
    const double chi = 2.0 - std::sqrt(2.0), a32 = 0.5;
    const double A[3][3] = {{0, 0, 0}, {chi, 0, 0}, {1.0 - a32, a32, 0}};
    const double B[3] = {0.5 - chi / 4.0, 0.5 - chi / 4.0, chi / 2.0};
    const double AT[3][3] = {{0, 0, 0}, {chi / 2.0, chi / 2.0, 0}, {B[0], B[1], B[2]}};
    for (int i = 0; i < 3; ++i) {
      b[i] = B[i];
      for (int j = 0; j < 3; ++j) {
        a[i][j] = A[i][j];
        at[i][j] = AT[i][j];
      }
    }
  }
};

// Block-partial dot products v_k . w for the NG vectors vec[0..NG) over
// the block's element range [lo, hi): each thread sums its elements in
// order, warps reduce by shuffles, the first warp adds the 8 warp sums (a
// fixed order, so results are deterministic).  Exactly NG FP64 FMAs per
// element: on GB300 these dot products are bound by the FP64 pipe, not by
// HBM, so no padded group slot is computed.  Block of 256 threads.
template <int NG>
__device__ __forceinline__ void block_dots(const double* const* vec, const double* __restrict__ w, int64_t lo,
                                           int64_t hi, double (*red)[8], double* __restrict__ out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const double* p[NG];
#pragma unroll
  for (int g = 0; g < NG; ++g) p[g] = vec[g];
  double s[NG];
#pragma unroll
  for (int g = 0; g < NG; ++g) s[g] = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const double wi = w[i];
#pragma unroll
    for (int g = 0; g < NG; ++g) s[g] += p[g][i] * wi;
  }
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    double t = s[g];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[g][wid] = t;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      double t = lane < 8 ? red[g][lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) out[g] = t;
    }
  }
  __syncthreads();
}

// the group of up to 8 vectors starting at k0 = 8 blockIdx.y (one group per
// block row of the grid); vec(k) gives the k-th vector, out(k0) the slots
template <typename VecOf, typename OutOf>
__device__ __forceinline__ void block_dots_group(int nvec, VecOf vec_of, const double* __restrict__ w, int64_t lo,
                                                 int64_t hi, OutOf out_of) {
  __shared__ double red[8][8];
  const int k0 = 8 * blockIdx.y;
  if (k0 < nvec) {
    const int ng = nvec - k0 < 8 ? nvec - k0 : 8;
    const double* vec[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) vec[g] = vec_of(k0 + (g < ng ? g : 0));
    double* out = out_of(k0);
    switch (ng) {
      case 8: block_dots<8>(vec, w, lo, hi, red, out); break;
      case 7: block_dots<7>(vec, w, lo, hi, red, out); break;
      case 6: block_dots<6>(vec, w, lo, hi, red, out); break;
      case 5: block_dots<5>(vec, w, lo, hi, red, out); break;
      case 4: block_dots<4>(vec, w, lo, hi, red, out); break;
      case 3: block_dots<3>(vec, w, lo, hi, red, out); break;
      case 2: block_dots<2>(vec, w, lo, hi, red, out); break;
      default: block_dots<1>(vec, w, lo, hi, red, out); break;
    }
  }
}

// w += sum_k c[k] V_k over element pairs (n even, V 16-byte aligned)
__device__ __forceinline__ void multiaxpy_pair(const double* __restrict__ V, int nvec, int64_t n,
                                               const double* __restrict__ c, double* __restrict__ w,
                                               int64_t i2) {
  double2 acc = reinterpret_cast<double2*>(w)[i2];
  int k = 0;
  for (; k + 4 <= nvec; k += 4) {
    double2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = reinterpret_cast<const double2*>(V + (int64_t)(k + u) * n)[i2];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      acc.x += c[k + u] * v[u].x;
      acc.y += c[k + u] * v[u].y;
    }
  }
  for (; k < nvec; ++k) {
    const double2 v = reinterpret_cast<const double2*>(V + (int64_t)k * n)[i2];
    acc.x += c[k] * v.x;
    acc.y += c[k] * v.y;
  }
  reinterpret_cast<double2*>(w)[i2] = acc;
}

__global__ void k_multidot(const double* __restrict__ V, int nvec, int64_t n, const double* __restrict__ w,
                           double* __restrict__ partial);
__global__ void k_reduce_partials(const double* __restrict__ partial, int nvec, int nblk, double* __restrict__ out);
__global__ void k_axpby(int64_t n, double a, const double* x, double b, const double* y, double* z);
__global__ void k_stage_predict(const double* __restrict__ q, int64_t n, StageCoefs c, double* __restrict__ rho,
                                double* __restrict__ mhat, double* __restrict__ ehat);
__global__ void k_primitives(const double* __restrict__ q, int64_t n, double gamma, double* __restrict__ u,
                             double* __restrict__ p);
__global__ void k_stage_state(const double* __restrict__ rho, const double* __restrict__ u,
                              const double* __restrict__ p, int64_t n, double gamma, double* __restrict__ y);
__global__ void k_final_update(double* __restrict__ q, int64_t n, StageCoefs c, const int* __restrict__ skip);
__global__ void k_picard_norms(const double* __restrict__ p0, const double* __restrict__ p1,
                               const double* __restrict__ u0, const double* __restrict__ u1, int64_t n,
                               double* __restrict__ partial);

int ensure_red(dg_mesh* m, Red* r);
Vmult make_vmult(SchurCtx* s);
Vmult make_vmult32(Schur32Ctx* s);
Vmult make_vmult_pairs(SchurDfCtx* s);
int prepare_pairs(dg_mesh* m, const ImplK& k, const double* rho, const double* plag, const double* ulag,
                  int penalty, cudaStream_t st, SchurDfCtx* out);
int prepare32(dg_mesh* m, const ImplK& k, const double* rho, const double* plag, const double* ulag, int penalty,
              cudaStream_t st, Schur32Ctx* out);
int prepare_rt(dg_mesh* m, const ImplK& k, const double* rho, const double* plag, const double* ulag, int penalty,
               cudaStream_t st);
int explicit_rt(dg_mesh* m, const dg_phys* ph, const double* q, double* fns, double* fs, cudaStream_t st);
int rhs_rt(dg_mesh* m, const ImplK& k, const double* rho, const double* plag, const double* ulag,
           const double* mhat, const double* ehat, double* rhs, cudaStream_t st);
int recover_rt(dg_mesh* m, const ImplK& k, const double* rho, const double* ulag, const double* mhat,
               const double* p, double* u, cudaStream_t st);

// vertical-line preconditioner (vline.cu): setup from the FP64 frozen
// coefficients that prepare_rt leaves (1/rho, h rho traces, penalty), then
// z = P^{-1} r as often as needed
int vline_setup(dg_mesh* m, const ImplK& k, const double* plag, int penalty, cudaStream_t st);
int vline_apply(dg_mesh* m, const double* r, double* z, cudaStream_t st);
// cell-block preconditioner (cellblock.cu): exact diagonal cell blocks of
// the scaled Schur operator, inverted in FP32
int cellblock_setup(dg_mesh* m, const ImplK& k, const double* plag, int penalty, cudaStream_t st);
int cellblock_apply(dg_mesh* m, const double* r, double* z, cudaStream_t st);
// the preconditioner of kind DG_PRECOND_* (setup records it in m->pc_kind)
int precond_setup(dg_mesh* m, int kind, const ImplK& k, const double* plag, int penalty, cudaStream_t st);
int precond_apply(dg_mesh* m, const double* r, double* z, cudaStream_t st);

// host-driven ARK2 step (any options) and the device-driven one (graph.cu)
int step_host(dg_mesh* m, const dg_phys* ph, double* q, double dt, const dg_step_opts* opts,
              dg_step_info* info, cudaStream_t st);
int step_graph(dg_mesh* m, const dg_phys* ph, double* q, double dt, const dg_step_opts* opts,
               dg_step_info* info, cudaStream_t st);

}  // namespace dg
