// Pieces of the Krylov solver and the ARK2 step shared by the host-driven
// step (solver.cu) and the device-driven step captured as a CUDA graph
// (graph.cu).
#pragma once

#include <cmath>

#include "engine.cuh"

namespace dg {

constexpr int RED_BLOCKS = 1024;   // partial sums per reduction (fixed order)
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
int prepare32(dg_mesh* m, const ImplK& k, const double* rho, const double* plag, const double* ulag, int penalty,
              cudaStream_t st, Schur32Ctx* out);
int prepare_rt(dg_mesh* m, const ImplK& k, const double* rho, const double* plag, const double* ulag, int penalty,
               cudaStream_t st);
int explicit_rt(dg_mesh* m, const dg_phys* ph, const double* q, double* fns, double* fs, cudaStream_t st);
int rhs_rt(dg_mesh* m, const ImplK& k, const double* rho, const double* plag, const double* ulag,
           const double* mhat, const double* ehat, double* rhs, cudaStream_t st);
int recover_rt(dg_mesh* m, const ImplK& k, const double* rho, const double* ulag, const double* mhat,
               const double* p, double* u, cudaStream_t st);

// host-driven ARK2 step (any options) and the device-driven one (graph.cu)
int step_host(dg_mesh* m, const dg_phys* ph, double* q, double dt, const dg_step_opts* opts,
              dg_step_info* info, cudaStream_t st);
int step_graph(dg_mesh* m, const dg_phys* ph, double* q, double dt, const dg_step_opts* opts,
               dg_step_info* info, cudaStream_t st);

}  // namespace dg
