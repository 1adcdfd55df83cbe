// GMRES on the scaled pressure Schur system, the Picard loop and the ARK2
// IMEX step (Section 3), with FP64 device reductions.
#include <cmath>
#include <vector>

#include "solver.cuh"

namespace dg {


// ---------------------------------------------------------------------------
// vector kernels (FP64)
// ---------------------------------------------------------------------------

// partial[b * nvec + k] = block b's share of V_k . w (contiguous chunk of
// elements per block column b, one group of 8 vectors per block row; launch
// grid (RED_BLOCKS, ceil(nvec / 8)) of 256 threads)
__global__ void k_multidot(const double* __restrict__ V, int nvec, int64_t n, const double* __restrict__ w,
                           double* __restrict__ partial) {
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  block_dots_group(
      nvec, [&](int k) { return V + (int64_t)k * n; }, w, lo, hi,
      [&](int k0) { return partial + (int64_t)blockIdx.x * nvec + k0; });
}

__global__ void k_reduce_partials(const double* __restrict__ partial, int nvec, int nblk, double* __restrict__ out) {
  __shared__ double red[256];
  const int k = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partial[b * nvec + k];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[k] = red[0];
}


// w += sum_k c_k V_k (one element per thread; any n)
__global__ void k_multiaxpy(const double* __restrict__ V, int nvec, int64_t n, Coefs c, double* __restrict__ w) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = w[i];
  for (int k = 0; k < nvec; ++k) acc += c.c[k] * V[(int64_t)k * n + i];
  w[i] = acc;
}

// the same over element pairs (n even, V and w 16-byte aligned): 16-byte loads
__global__ void k_multiaxpy2(const double* __restrict__ V, int nvec, int64_t n, Coefs c, double* __restrict__ w) {
  int64_t i2 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (2 * i2 >= n) return;
  multiaxpy_pair(V, nvec, n, c.c, w, i2);
}

static void launch_multiaxpy(dg_mesh* m, const double* V, int nvec, int64_t n, const Coefs& c, double* w,
                             cudaStream_t st) {
  if (n % 2 == 0 && ((uintptr_t)w & 15) == 0 && ((uintptr_t)V & 15) == 0)
    DG_RUN(m, K_MULTIAXPY, st, k_multiaxpy2<<<grid_for(n / 2, 256), 256, 0, st>>>(V, nvec, n, c, w));
  else
    DG_RUN(m, K_MULTIAXPY, st, k_multiaxpy<<<grid_for(n, 256), 256, 0, st>>>(V, nvec, n, c, w));
}

__global__ void k_axpby(int64_t n, double a, const double* x, double b, const double* y, double* z) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) z[i] = a * x[i] + b * y[i];
}

__global__ void k_scale(int64_t n, double a, double* __restrict__ x) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] *= a;
}


// stage predictors: rho_l = rho^n + dt sum a F_NS,rho;
// m_hat = m^n + dt sum (a F_NS,m + at F_S,m); e_hat likewise
__global__ void k_stage_predict(const double* __restrict__ q, int64_t n, StageCoefs c, double* __restrict__ rho,
                                double* __restrict__ mhat, double* __restrict__ ehat) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double r = 0, m0 = 0, m1 = 0, m2 = 0, e = 0;
#pragma unroll
  for (int s = 0; s < 3; ++s) {   // static indices into c (no local copy)
    if (s >= c.nst) break;
    const double a = c.a[s], at = c.at[s];
    const double* F = c.fns[s];
    const double* G = c.fs[s];
    r += a * F[i];
    m0 += a * F[n + i] + at * G[i];
    m1 += a * F[2 * n + i] + at * G[n + i];
    m2 += a * F[3 * n + i] + at * G[2 * n + i];
    e += a * F[4 * n + i] + at * G[3 * n + i];
  }
  rho[i] = q[i] + c.dt * r;
  mhat[i] = q[n + i] + c.dt * m0;
  mhat[n + i] = q[2 * n + i] + c.dt * m1;
  mhat[2 * n + i] = q[3 * n + i] + c.dt * m2;
  ehat[i] = q[4 * n + i] + c.dt * e;
}

// nodal u = m / rho, p = (gamma - 1)(E - m.u / 2)
__global__ void k_primitives(const double* __restrict__ q, int64_t n, double gamma, double* __restrict__ u,
                             double* __restrict__ p) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double ir = 1.0 / q[i];
  const double u0 = q[n + i] * ir, u1 = q[2 * n + i] * ir, u2 = q[3 * n + i] * ir;
  u[i] = u0;
  u[n + i] = u1;
  u[2 * n + i] = u2;
  p[i] = (gamma - 1.0) * (q[4 * n + i] - 0.5 * (q[n + i] * u0 + q[2 * n + i] * u1 + q[3 * n + i] * u2));
}

// stage state: m = rho u, E = p / (gamma - 1) + rho |u|^2 / 2
__global__ void k_stage_state(const double* __restrict__ rho, const double* __restrict__ u,
                              const double* __restrict__ p, int64_t n, double gamma, double* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double r = rho[i], u0 = u[i], u1 = u[n + i], u2 = u[2 * n + i];
  y[i] = r;
  y[n + i] = r * u0;
  y[2 * n + i] = r * u1;
  y[3 * n + i] = r * u2;
  y[4 * n + i] = p[i] / (gamma - 1.0) + 0.5 * r * (u0 * u0 + u1 * u1 + u2 * u2);
}

// q += dt sum_l b_l (F_NS,l + F_S,l)
// (skipped when *skip != 0: the device-driven step's error status)
__global__ void k_final_update(double* __restrict__ q, int64_t n, StageCoefs c, const int* __restrict__ skip) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n || (skip && *skip)) return;
  double acc[5] = {0, 0, 0, 0, 0};
#pragma unroll
  for (int s = 0; s < 3; ++s) {   // static indices into c (no local copy)
    if (s >= c.nst) break;
    const double b = c.a[s];
    const double* F = c.fns[s];
    const double* G = c.fs[s];
    acc[0] += b * F[i];
    for (int k = 1; k < 5; ++k) acc[k] += b * (F[k * n + i] + G[(k - 1) * n + i]);
  }
  for (int k = 0; k < 5; ++k) q[k * n + i] += c.dt * acc[k];
}

// four sums for the Picard test: |p1-p0|^2, |p1|^2, |u1-u0|^2, |u1|^2
__global__ void k_picard_norms(const double* __restrict__ p0, const double* __restrict__ p1,
                               const double* __restrict__ u0, const double* __restrict__ u1, int64_t n,
                               double* __restrict__ partial) {
  __shared__ double red[4][256];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  double s[4] = {0, 0, 0, 0};
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const double dp = p1[i] - p0[i];
    s[0] += dp * dp;
    s[1] += p1[i] * p1[i];
    for (int c = 0; c < 3; ++c) {
      const double a = u1[c * n + i], du = a - u0[c * n + i];
      s[2] += du * du;
      s[3] += a * a;
    }
  }
  for (int k = 0; k < 4; ++k) red[k][threadIdx.x] = s[k];
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int k = 0; k < 4; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) partial[blockIdx.x * 4 + k] = red[k][0];
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------


int ensure_red(dg_mesh* m, Red* r) {
  int rc = m->red.ensure(sizeof(double) * (RED_BLOCKS * (MAX_RESTART + 1) + (MAX_RESTART + 1)));
  if (rc) return rc;
  r->partial = m->red.as<double>();
  r->out = r->partial + RED_BLOCKS * (MAX_RESTART + 1);
  return DG_OK;
}

// host <- V[0..nvec)^T w  (synchronises the stream)
static int dots(dg_mesh* m, const Red& r, const double* V, int nvec, int64_t n, const double* w,
                double* host, cudaStream_t st) {
  DG_RUN(m, K_MULTIDOT, st, k_multidot<<<dim3(RED_BLOCKS, (nvec + 7) / 8), 256, 0, st>>>(V, nvec, n, w, r.partial));
  DG_RUN(m, K_REDUCE, st, k_reduce_partials<<<nvec, 256, 0, st>>>(r.partial, nvec, RED_BLOCKS, r.out));
  DG_LAUNCH_CHECK("reduction");
  DG_CUDA(cudaMemcpyAsync(host, r.out, sizeof(double) * nvec, cudaMemcpyDeviceToHost, st));
  DG_CUDA(cudaStreamSynchronize(st));
  return DG_OK;
}


// Restarted GMRES(m), classical Gram-Schmidt applied twice, Givens rotations.
static int gmres(dg_mesh* m, const Vmult& A, const double* b, double* x, double rtol, int restart, int maxit,
                 dg_gmres_info* info, cudaStream_t st, bool x_is_zero = false, bool pc = false) {
  const int64_t n = m->N;
  if (restart < 1 || restart > MAX_RESTART || maxit < 0 || !(rtol >= 0.0)) {
    set_error("gmres: restart must be in 1..%d, maxit >= 0, rtol >= 0", MAX_RESTART);
    return DG_ERR_ARG;
  }
  int rc;
  if ((rc = m->gm_V.ensure(sizeof(double) * (size_t)(restart + 1) * n)) != DG_OK) return rc;
  if ((rc = m->gm_work.ensure(sizeof(double) * (size_t)n)) != DG_OK) return rc;
  // right preconditioning in flexible form: Z_j = P^{-1} V_j is kept and x
  // gains Z y, so the update matches the Arnoldi relation A Z = V H even
  // though P^{-1} (FP32 factors) is only accurate to rounding; residuals
  // are those of A x = b itself
  // (one column more than restart: the device-driven solver keeps the
  // current preconditioned vector there, and sizes its workspace by a
  // host-driven step)
  if (pc && (rc = m->gm_pc.ensure(sizeof(double) * (size_t)(restart + 1) * n)) != DG_OK) return rc;
  double* Z = pc ? m->gm_pc.as<double>() : nullptr;
  Red red;
  if ((rc = ensure_red(m, &red)) != DG_OK) return rc;
  double* V = m->gm_V.as<double>();
  double* tmp = m->gm_work.as<double>();
  const unsigned gb = grid_for(n, 256);
  double bn2;
  if ((rc = dots(m, red, b, 1, n, b, &bn2, st)) != DG_OK) return rc;
  const double bnorm = std::sqrt(bn2);
  if (!std::isfinite(bnorm)) {
    set_error("gmres: non-finite right-hand side");
    return DG_ERR_NONFINITE;
  }
  if (bnorm == 0.0) {
    DG_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    if (info) {
      info->iters = 0;
      info->relres = 0.0;
    }
    return DG_OK;
  }
  std::vector<double> H((restart + 1) * restart), cs(restart), sn(restart), g(restart + 1), h1(restart + 1),
      h2(restart + 1), y(restart);
  auto Hij = [&](int i, int j) -> double& { return H[i * restart + j]; };
  int it = 0;
  double relres = 0.0;
  while (true) {
    if (x_is_zero && it == 0) {
      DG_CUDA(cudaMemcpyAsync(V, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    } else {
      if ((rc = A(x, tmp, st)) != DG_OK) return rc;
      DG_RUN(m, K_VEC, st, k_axpby<<<gb, 256, 0, st>>>(n, 1.0, b, -1.0, tmp, V));
    }
    double b2;
    if ((rc = dots(m, red, V, 1, n, V, &b2, st)) != DG_OK) return rc;
    const double beta = std::sqrt(b2);
    if (!std::isfinite(beta)) {
      set_error("gmres: non-finite residual");
      return DG_ERR_NONFINITE;
    }
    relres = beta / bnorm;
    if (beta <= rtol * bnorm || it >= maxit) {
      if (info) {
        info->iters = it;
        info->relres = relres;
      }
      if (beta <= rtol * bnorm) return DG_OK;
      set_error("gmres: %d iterations, relative residual %.3e > %.3e", it, relres, rtol);
      return DG_ERR_NOT_CONVERGED;
    }
    DG_RUN(m, K_VEC, st, k_scale<<<gb, 256, 0, st>>>(n, 1.0 / beta, V));
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jused = 0;
    for (int j = 0; j < restart; ++j) {
      double* vj = V + (int64_t)j * n;
      double* w = V + (int64_t)(j + 1) * n;
      if (pc) {
        double* zj = Z + (int64_t)j * n;
        if ((rc = precond_apply(m, vj, zj, st)) != DG_OK) return rc;
        if ((rc = A(zj, w, st)) != DG_OK) return rc;
      } else if ((rc = A(vj, w, st)) != DG_OK) {
        return rc;
      }
      // classical Gram-Schmidt with a re-orthogonalisation test: one pass
      // gives V^T w and |w|^2 together (w is stored right after V_j); a
      // second pass runs only when the projection cancelled w down to
      // |w'| < 1e-3 |w|, where one pass would lose more than ~1e3 eps of
      // orthogonality.  (The scaled Schur operator is close to the identity,
      // so w is dominated by its V_j component and a stricter threshold
      // would re-orthogonalise every step.)
      Coefs c;
      if ((rc = dots(m, red, V, j + 2, n, w, h1.data(), st)) != DG_OK) return rc;
      double proj = 0.0;
      for (int k = 0; k <= j; ++k) {
        c.c[k] = -h1[k];
        proj += h1[k] * h1[k];
        Hij(k, j) = h1[k];
      }
      launch_multiaxpy(m, V, j + 1, n, c, w, st);
      double w2 = h1[j + 1] - proj;
      if (!(w2 > 1e-6 * h1[j + 1])) {
        if ((rc = dots(m, red, V, j + 2, n, w, h2.data(), st)) != DG_OK) return rc;
        proj = 0.0;
        for (int k = 0; k <= j; ++k) {
          c.c[k] = -h2[k];
          proj += h2[k] * h2[k];
          Hij(k, j) += h2[k];
        }
        launch_multiaxpy(m, V, j + 1, n, c, w, st);
        w2 = h2[j + 1] - proj;
      }
      if (w2 < 0.0) w2 = 0.0;
      const double hn = std::sqrt(w2);
      if (!std::isfinite(hn)) {
        set_error("gmres: non-finite Krylov vector");
        return DG_ERR_NONFINITE;
      }
      Hij(j + 1, j) = hn;
      if (hn > 0.0) DG_RUN(m, K_VEC, st, k_scale<<<gb, 256, 0, st>>>(n, 1.0 / hn, w));
      for (int k = 0; k < j; ++k) {
        const double t = cs[k] * Hij(k, j) + sn[k] * Hij(k + 1, j);
        Hij(k + 1, j) = -sn[k] * Hij(k, j) + cs[k] * Hij(k + 1, j);
        Hij(k, j) = t;
      }
      const double den = std::hypot(Hij(j, j), Hij(j + 1, j));
      cs[j] = Hij(j, j) / den;
      sn[j] = Hij(j + 1, j) / den;
      Hij(j, j) = den;
      Hij(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++it;
      jused = j + 1;
      if (std::fabs(g[j + 1]) <= rtol * bnorm || it >= maxit) break;
    }
    for (int i = jused - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < jused; ++k) s -= Hij(i, k) * y[k];
      y[i] = s / Hij(i, i);
    }
    Coefs c;
    for (int k = 0; k < jused; ++k) c.c[k] = y[k];
    launch_multiaxpy(m, pc ? Z : V, jused, n, c, x, st);
    DG_LAUNCH_CHECK("gmres update");
  }
}


template <int D, int NN>
static int schur_vmult_fn(void* self, const double* x, double* y, cudaStream_t st) {
  SchurCtx* s = static_cast<SchurCtx*>(self);
  return Engine<double, D, NN>::vmult(s->m, s->k, s->rho, s->plag, s->penalty, x, y, st);
}

Vmult make_vmult(SchurCtx* s) {
  Vmult v{nullptr, s};
  DG_DISPATCH(s->m, v.fn = &schur_vmult_fn<D_, N_>);
  return v;
}

// ---------------------------------------------------------------------------
// mixed precision: FP32 Schur vmult behind an FP64 interface
// ---------------------------------------------------------------------------

__global__ void k_d2f(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

__global__ void k_f2d(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}


template <int D, int NN>
static int schur32_vmult_fn(void* self, const double* x, double* y, cudaStream_t st) {
  Schur32Ctx* s = static_cast<Schur32Ctx*>(self);
  dg_mesh* m = s->m;
  const unsigned gb = grid_for(m->N, 256);
  DG_RUN(m, K_VEC, st, k_d2f<<<gb, 256, 0, st>>>(x, s->x32, m->N));
  int rc = Engine<float, D, NN>::vmult(m, s->k, s->rho, s->plag, s->penalty, s->x32, s->y32, st);
  if (rc != DG_OK) return rc;
  DG_RUN(m, K_VEC, st, k_f2d<<<gb, 256, 0, st>>>(s->y32, y, m->N));
  DG_LAUNCH_CHECK("fp32 vmult casts");
  return DG_OK;
}

// FP32 copies of the frozen coefficients and their face data (h rho traces,
// implicit Rusanov lambda) for the FP32 vmult.
int prepare32(dg_mesh* m, const ImplK& k, const double* rho, const double* plag, const double* ulag,
                     int penalty, cudaStream_t st, Schur32Ctx* out) {
  int rc;
  if ((rc = ensure_fp32_geometry(m)) != DG_OK) return rc;
  const int64_t n = m->N;
  if ((rc = m->c32.ensure(sizeof(float) * (5 * n + m->E))) != DG_OK) return rc;
  if ((rc = m->ir32.ensure(sizeof(float) * 2 * n)) != DG_OK) return rc;
  float* c = m->c32.as<float>();
  const unsigned gb = grid_for(n, 256), gb3 = grid_for(3 * n, 256);
  DG_RUN(m, K_VEC, st, k_d2f<<<gb, 256, 0, st>>>(rho, c, n));
  DG_RUN(m, K_VEC, st, k_d2f<<<gb, 256, 0, st>>>(plag, c + n, n));
  DG_RUN(m, K_VEC, st, k_d2f<<<gb3, 256, 0, st>>>(ulag, c + 2 * n, 3 * n));
  DG_LAUNCH_CHECK("fp32 coefficient casts");
  rc = DG_ERR_UNSUPPORTED;
  DG_DISPATCH(m, rc = (Engine<float, D_, N_>::prepare(m, k, c, c + n, c + 2 * n, penalty, st)));
  if (rc != DG_OK) return rc;
  *out = Schur32Ctx{m, k, c, c + n, penalty, m->ir32.as<float>(), m->ir32.as<float>() + n};
  if (k.fcell) {   // FP32 copy of the per-cell Coriolis parameter after the coefficients
    float* fc = c + 5 * n;
    DG_RUN(m, K_VEC, st, k_d2f<<<grid_for(m->E, 256), 256, 0, st>>>(k.fcell, fc, m->E));
    DG_LAUNCH_CHECK("fp32 coriolis cast");
    out->k.fcell32 = fc;
  }
  return DG_OK;
}

Vmult make_vmult32(Schur32Ctx* s) {
  Vmult v{nullptr, s};
  DG_DISPATCH(s->m, v.fn = &schur32_vmult_fn<D_, N_>);
  return v;
}

template <int D, int NN>
static int schur_pairs_vmult_fn(void* self, const double* x, double* y, cudaStream_t st) {
  SchurDfCtx* s = static_cast<SchurDfCtx*>(self);
  dg_mesh* m = s->m;
  int rc;
  if ((rc = to_pairs(m, x, s->xdf, m->N, st)) != DG_OK) return rc;
  if ((rc = Engine<df64, D, NN>::vmult(m, s->k, s->rho, s->plag, s->penalty, s->xdf, s->ydf, st)) != DG_OK)
    return rc;
  return from_pairs(m, s->ydf, y, m->N, st);
}

// Pair copies of the frozen coefficients and their face data for the
// DG_PAIRS vmult (the FP64 ones stay for the right-hand side and recovery).
int prepare_pairs(dg_mesh* m, const ImplK& k, const double* rho, const double* plag, const double* ulag,
                  int penalty, cudaStream_t st, SchurDfCtx* out) {
  int rc;
  if ((rc = ensure_pairs_geometry(m, st)) != DG_OK) return rc;
  const int64_t n = m->N;
  if ((rc = m->cdf.ensure(sizeof(df64) * 5 * n)) != DG_OK) return rc;
  if ((rc = m->irdf.ensure(sizeof(df64) * 2 * n)) != DG_OK) return rc;
  df64* c = m->cdf.as<df64>();
  if ((rc = to_pairs(m, rho, c, n, st)) != DG_OK) return rc;
  if ((rc = to_pairs(m, plag, c + n, n, st)) != DG_OK) return rc;
  if ((rc = to_pairs(m, ulag, c + 2 * n, 3 * n, st)) != DG_OK) return rc;
  rc = DG_ERR_UNSUPPORTED;
  DG_DISPATCH(m, rc = (Engine<df64, D_, N_>::prepare(m, k, c, c + n, c + 2 * n, penalty, st)));
  if (rc != DG_OK) return rc;
  *out = SchurDfCtx{m, k, c, c + n, penalty, m->irdf.as<df64>(), m->irdf.as<df64>() + n};
  return DG_OK;
}

Vmult make_vmult_pairs(SchurDfCtx* s) {
  Vmult v{nullptr, s};
  DG_DISPATCH(s->m, v.fn = &schur_pairs_vmult_fn<D_, N_>);
  return v;
}

int schur_vmult_pairs(dg_mesh* m, const ImplK& k, const double* rho, const double* plag, const double* ulag,
                      int penalty, const double* x, double* y, cudaStream_t st) {
  SchurDfCtx sc;
  int rc = prepare_pairs(m, k, rho, plag, ulag, penalty, st, &sc);
  if (rc != DG_OK) return rc;
  Vmult A = make_vmult_pairs(&sc);
  if (!A.fn) return DG_ERR_UNSUPPORTED;
  return A(x, y, st);
}

int schur_vmult_mixed(dg_mesh* m, const ImplK& k, const double* rho, const double* plag, const double* ulag,
                      int penalty, const double* x, double* y, cudaStream_t st) {
  Schur32Ctx sc;
  int rc = prepare32(m, k, rho, plag, ulag, penalty, st, &sc);
  if (rc != DG_OK) return rc;
  Vmult A = make_vmult32(&sc);
  if (!A.fn) return DG_ERR_UNSUPPORTED;
  return A(x, y, st);
}

// Iterative refinement: FP64 residual r = b - A64 x, correction from GMRES
// on the FP32 operator (FP64 basis, orthogonalisation and reductions) to
// relative residual inner_rtol, x += d; until ||r|| <= rtol ||b||.
static int gmres_ir(dg_mesh* m, const Vmult& A64, const Vmult& A32, const double* b, double* x, double rtol,
                    int restart, int maxit, double inner_rtol, dg_gmres_info* info, cudaStream_t st,
                    bool pc = false) {
  const int64_t n = m->N;
  int rc;
  if ((rc = m->irw.ensure(sizeof(double) * 2 * n)) != DG_OK) return rc;
  Red red;
  if ((rc = ensure_red(m, &red)) != DG_OK) return rc;
  double* r = m->irw.as<double>();
  double* d = r + n;
  const unsigned gb = grid_for(n, 256);
  if (!(inner_rtol > 0.0)) inner_rtol = 1e-4;
  double bn2;
  if ((rc = dots(m, red, b, 1, n, b, &bn2, st)) != DG_OK) return rc;
  const double bnorm = std::sqrt(bn2);
  if (!std::isfinite(bnorm)) {
    set_error("gmres (mixed): non-finite right-hand side");
    return DG_ERR_NONFINITE;
  }
  dg_gmres_info out{0, 0.0, 0};
  if (bnorm == 0.0) {
    DG_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    if (info) *info = out;
    return DG_OK;
  }
  for (int sweep = 0;; ++sweep) {
    if ((rc = A64(x, r, st)) != DG_OK) return rc;
    DG_RUN(m, K_VEC, st, k_axpby<<<gb, 256, 0, st>>>(n, 1.0, b, -1.0, r, r));
    double r2;
    if ((rc = dots(m, red, r, 1, n, r, &r2, st)) != DG_OK) return rc;
    const double rn = std::sqrt(r2);
    if (!std::isfinite(rn)) {
      set_error("gmres (mixed): non-finite residual");
      return DG_ERR_NONFINITE;
    }
    out.relres = rn / bnorm;
    out.refinements = sweep;
    if (rn <= rtol * bnorm) break;
    if (out.iters >= maxit || sweep >= 60) {
      if (info) *info = out;
      set_error("gmres (mixed): %d inner iterations, %d sweeps, relative residual %.3e > %.3e", out.iters,
                sweep, out.relres, rtol);
      return DG_ERR_NOT_CONVERGED;
    }
    // the inner solve only has to beat the FP32 operator's accuracy
    const double tol_in = std::max(inner_rtol, 0.5 * rtol * bnorm / rn);
    DG_CUDA(cudaMemsetAsync(d, 0, sizeof(double) * n, st));
    dg_gmres_info gi{0, 0.0, 0};
    rc = gmres(m, A32, r, d, tol_in, restart, maxit - out.iters, &gi, st, true, pc);
    if (rc != DG_OK && rc != DG_ERR_NOT_CONVERGED) return rc;
    out.iters += gi.iters;
    DG_RUN(m, K_VEC, st, k_axpby<<<gb, 256, 0, st>>>(n, 1.0, x, 1.0, d, x));
    DG_LAUNCH_CHECK("refinement update");
  }
  if (info) *info = out;
  return DG_OK;
}

int prepare_rt(dg_mesh* m, const ImplK& k, const double* rho, const double* plag, const double* ulag,
                      int penalty,
                      cudaStream_t st) {
  DG_DISPATCH(m, return (Engine<double, D_, N_>::prepare(m, k, rho, plag, ulag, penalty, st)));
  return DG_ERR_UNSUPPORTED;
}

int explicit_rt(dg_mesh* m, const dg_phys* ph, const double* q, double* fns, double* fs, cudaStream_t st) {
  PhysK k{ph->gamma, ph->g, ph->f, ph->f_cell, ph->lambda_min};
  int rc = DG_ERR_UNSUPPORTED;
  if (ph->precision == DG_MIXED_EXPLICIT && m->bg_set)
    rc = explicit_mixed(m, k, q, fns, fs, st);
  else
    DG_DISPATCH(m, rc = (Engine<double, D_, N_>::explicit_rates(m, k, q, fns, fs, st)));
  if (rc != DG_OK) return rc;
  return sponge_rt(m, q, fns, st);
}

int rhs_rt(dg_mesh* m, const ImplK& k, const double* rho, const double* plag, const double* ulag,
                  const double* mhat, const double* ehat, double* rhs, cudaStream_t st) {
  DG_DISPATCH(m, return (Engine<double, D_, N_>::schur_rhs(m, k, rho, plag, ulag, mhat, ehat, rhs, st)));
  return DG_ERR_UNSUPPORTED;
}

int recover_rt(dg_mesh* m, const ImplK& k, const double* rho, const double* ulag, const double* mhat,
                      const double* p, double* u, cudaStream_t st) {
  DG_DISPATCH(m, return (Engine<double, D_, N_>::recover(m, k, rho, ulag, mhat, p, u, st)));
  return DG_ERR_UNSUPPORTED;
}

static int check_phys(const dg_phys* ph, const char* who) {
  if (!ph || !(ph->gamma > 1.0) || (ph->variant != DG_R1 && ph->variant != DG_R2) || !(ph->lambda_min >= 0.0)) {
    set_error("%s: invalid physics (gamma > 1, variant R1/R2, lambda_min >= 0)", who);
    return DG_ERR_ARG;
  }
  if (ph->precision != DG_FP64 && ph->precision != DG_MIXED && ph->precision != DG_MIXED_EXPLICIT &&
      ph->precision != DG_PAIRS) {
    set_error("%s: precision must be DG_FP64, DG_MIXED, DG_MIXED_EXPLICIT or DG_PAIRS", who);
    return DG_ERR_ARG;
  }
  return DG_OK;
}

}  // namespace dg

using namespace dg;

extern "C" {

int dg_gmres_solve(dg_ctx* ctx, const dg_mesh* mesh, const dg_phys* ph, const dg_implicit_coeffs* cf,
                   const double* b, double* x, const dg_gmres_opts* opts, dg_gmres_info* info, void* stream) {
  if (!ctx || !mesh || !cf || !cf->rho || !cf->p_lag || !cf->u_lag || !b || !x || !opts) {
    set_error("dg_gmres_solve: NULL argument");
    return DG_ERR_ARG;
  }
  int rc = check_phys(ph, "dg_gmres_solve");
  if (rc) return rc;
  dg_mesh* m = const_cast<dg_mesh*>(mesh);
  cudaStream_t st = (cudaStream_t)stream;
  if (opts->precond < DG_PRECOND_NONE || opts->precond > DG_PRECOND_CELL) {
    set_error("dg_gmres_solve: precond must be DG_PRECOND_NONE, DG_PRECOND_VLINE or DG_PRECOND_CELL");
    return DG_ERR_ARG;
  }
  const bool pc = opts->precond != DG_PRECOND_NONE;
  if (pc && m->gll) {
    set_error("dg_gmres_solve: the preconditioners are not implemented for Gauss-Lobatto nodes");
    return DG_ERR_UNSUPPORTED;
  }
  ImplK k = impl_consts(ph, cf->a_dt);
  if ((rc = prepare_rt(m, k, cf->rho, cf->p_lag, cf->u_lag, ph->penalty, st)) != DG_OK) return rc;
  if (pc && (rc = precond_setup(m, opts->precond, k, cf->p_lag, ph->penalty, st)) != DG_OK) return rc;
  SchurCtx sc{m, k, cf->rho, cf->p_lag, ph->penalty};
  Vmult A = make_vmult(&sc);
  if (!A.fn) return DG_ERR_UNSUPPORTED;
  if (ph->precision == DG_PAIRS) {
    SchurDfCtx sdf;
    if ((rc = prepare_pairs(m, k, cf->rho, cf->p_lag, cf->u_lag, ph->penalty, st, &sdf)) != DG_OK) return rc;
    if (info) info->refinements = 0;
    return gmres(m, make_vmult_pairs(&sdf), b, x, opts->rtol, opts->restart, opts->maxit, info, st, false, pc);
  }
  if (ph->precision != DG_FP64) {
    Schur32Ctx sc32;
    if ((rc = prepare32(m, k, cf->rho, cf->p_lag, cf->u_lag, ph->penalty, st, &sc32)) != DG_OK) return rc;
    Vmult A32 = make_vmult32(&sc32);
    return gmres_ir(m, A, A32, b, x, opts->rtol, opts->restart, opts->maxit, opts->inner_rtol, info, st, pc);
  }
  if (info) info->refinements = 0;
  return gmres(m, A, b, x, opts->rtol, opts->restart, opts->maxit, info, st, false, pc);
}

int imex_ark2_step(dg_ctx* ctx, const dg_mesh* mesh, const dg_phys* ph, double* q, double dt,
                   const dg_step_opts* opts, dg_step_info* info, void* stream) {
  if (!ctx || !mesh || !q || !opts) {
    set_error("imex_ark2_step: NULL argument");
    return DG_ERR_ARG;
  }
  int rc = check_phys(ph, "imex_ark2_step");
  if (rc) return rc;
  if (!(dt > 0.0) || opts->picard_maxit < 1 || opts->picard_fixed < 0) {
    set_error("imex_ark2_step: dt > 0, picard_maxit >= 1, picard_fixed >= 0 required");
    return DG_ERR_ARG;
  }
  if (opts->gmres.restart < 1 || opts->gmres.restart > MAX_RESTART || opts->gmres.maxit < 0 ||
      !(opts->gmres.rtol >= 0.0)) {
    set_error("imex_ark2_step: gmres restart must be in 1..%d, maxit >= 0, rtol >= 0", MAX_RESTART);
    return DG_ERR_ARG;
  }
  if (opts->gmres.precond < DG_PRECOND_NONE || opts->gmres.precond > DG_PRECOND_CELL) {
    set_error("imex_ark2_step: gmres precond must be DG_PRECOND_NONE, DG_PRECOND_VLINE or DG_PRECOND_CELL");
    return DG_ERR_ARG;
  }
  dg_mesh* m = const_cast<dg_mesh*>(mesh);
  cudaStream_t st = (cudaStream_t)stream;
  if (m->nFar > 0 && ph->precision == DG_MIXED_EXPLICIT) {
    set_error("imex_ark2_step: DG_MIXED_EXPLICIT is not implemented with far-field faces");
    return DG_ERR_UNSUPPORTED;
  }
  if (m->gll && (opts->graph || opts->gmres.precond != DG_PRECOND_NONE || ph->precision == DG_MIXED_EXPLICIT ||
                 m->sponge_set)) {
    set_error("imex_ark2_step: Gauss-Lobatto nodes support the host-driven, unpreconditioned step in DG_FP64, "
              "DG_MIXED or DG_PAIRS only");
    return DG_ERR_UNSUPPORTED;
  }
  if (opts->graph) return step_graph(m, ph, q, dt, opts, info, st);
  return step_host(m, ph, q, dt, opts, info, st);
}

}  // extern "C"

namespace dg {

// Stage state on a Gauss-Lobatto mesh: rho u = M^{-1} A u and rho E =
// M^{-1}(D p + k(u)) are pointwise at the Gauss-Legendre points, so (rho, u,
// p) go to the GL basis, k_stage_state runs there, and y comes back.
static int stage_state_gll(dg_mesh* m, const double* rho, const double* u, const double* p, double gamma,
                           double* y, cudaStream_t st) {
  const int64_t n = m->N;
  double* g = gl_scratch(m);
  if (!g) return DG_ERR_OOM;
  int rc;
  if ((rc = gl_basis(m, rho, g, 1, true, st)) != DG_OK) return rc;
  if ((rc = gl_basis(m, u, g + n, 3, true, st)) != DG_OK) return rc;
  if ((rc = gl_basis(m, p, g + 4 * n, 1, true, st)) != DG_OK) return rc;
  DG_RUN(m, K_STAGE, st, k_stage_state<<<grid_for(n, 256), 256, 0, st>>>(g, g + n, g + 4 * n, n, gamma, y));
  return gl_basis(m, y, y, 5, false, st);
}

int step_host(dg_mesh* m, const dg_phys* ph, double* q, double dt, const dg_step_opts* opts,
              dg_step_info* info, cudaStream_t st) {
  int rc;
  const int64_t n = m->N;
  const Ark2 tab;
  const auto& a = tab.a;
  const auto& at = tab.at;
  const auto& bw = tab.b;
  const bool pc = opts->gmres.precond != DG_PRECOND_NONE;
  // workspace: F_NS x3 (5n), F_S x3 (4n), y (5n), rho, mhat (3n), ehat, u, unew (3n each), p, pnew, rhs
  if ((rc = m->fns.ensure(sizeof(double) * 15 * n)) != DG_OK) return rc;
  if ((rc = m->fs.ensure(sizeof(double) * 12 * n)) != DG_OK) return rc;
  if ((rc = m->st.ensure(sizeof(double) * 19 * n)) != DG_OK) return rc;
  Red red;
  if ((rc = ensure_red(m, &red)) != DG_OK) return rc;
  double* Fns[3] = {m->fns.as<double>(), m->fns.as<double>() + 5 * n, m->fns.as<double>() + 10 * n};
  double* Fs[3] = {m->fs.as<double>(), m->fs.as<double>() + 4 * n, m->fs.as<double>() + 8 * n};
  double* w = m->st.as<double>();
  double* y = w;
  double* rho = w + 5 * n;
  double* mhat = w + 6 * n;
  double* ehat = w + 9 * n;
  double* u = w + 10 * n;
  double* unew = w + 13 * n;
  double* p = w + 16 * n;
  double* pnew = w + 17 * n;
  double* rhs = w + 18 * n;
  const unsigned gb = grid_for(n, 256);
  dg_step_info inf{};
  // FP32 explicit operator without a background: the rates of the later
  // stages are increments about the step's start state q, whose FP64 rates
  // are those of the first stage
  const bool incr = ph->precision == DG_MIXED_EXPLICIT && !m->bg_set;
  const PhysK pk{ph->gamma, ph->g, ph->f, ph->f_cell, ph->lambda_min};
  if ((rc = explicit_rt(m, ph, q, Fns[0], Fs[0], st)) != DG_OK) return rc;
  if (incr && (rc = increment_begin(m, ph->gamma, q, st)) != DG_OK) return rc;
  const double* yprev = q;
  for (int l = 1; l <= 2; ++l) {
    const double adt = at[l][l] * dt;
    StageCoefs sc{};
    sc.nst = l;
    sc.dt = dt;
    for (int s = 0; s < l; ++s) {
      sc.fns[s] = Fns[s];
      sc.fs[s] = Fs[s];
      sc.a[s] = a[l][s];
      sc.at[s] = at[l][s];
    }
    DG_RUN(m, K_STAGE, st, k_stage_predict<<<gb, 256, 0, st>>>(q, n, sc, rho, mhat, ehat));
    DG_RUN(m, K_STAGE, st, k_primitives<<<gb, 256, 0, st>>>(yprev, n, ph->gamma, u, p));
    DG_LAUNCH_CHECK("stage predictors");
    ImplK k = impl_consts(ph, adt);
    const int kmax = opts->picard_fixed > 0 ? opts->picard_fixed : opts->picard_maxit;
    int kk = 0;
    for (; kk < kmax; ++kk) {
      if ((rc = prepare_rt(m, k, rho, p, u, ph->penalty, st)) != DG_OK) return rc;
      // the preconditioner is factored once per stage, from the first Picard
      // iterate's coefficients: the flexible GMRES needs only an
      // approximate inverse, and the later iterates move the coefficients
      // too little to change the iteration counts (measured: same counts,
      // 4-12 % faster steps than refactoring every Picard iteration)
      if (pc && kk == 0 && (rc = precond_setup(m, opts->gmres.precond, k, p, ph->penalty, st)) != DG_OK) return rc;
      if ((rc = rhs_rt(m, k, rho, p, u, mhat, ehat, rhs, st)) != DG_OK) return rc;
      DG_CUDA(cudaMemcpyAsync(pnew, p, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
      SchurCtx schur{m, k, rho, p, ph->penalty};
      Vmult A = make_vmult(&schur);
      dg_gmres_info gi{};
      if (ph->precision == DG_PAIRS) {
        SchurDfCtx sdf;
        if ((rc = prepare_pairs(m, k, rho, p, u, ph->penalty, st, &sdf)) != DG_OK) return rc;
        rc = gmres(m, make_vmult_pairs(&sdf), rhs, pnew, opts->gmres.rtol, opts->gmres.restart, opts->gmres.maxit,
                   &gi, st, false, pc);
      } else if (ph->precision != DG_FP64) {
        Schur32Ctx sc32;
        if ((rc = prepare32(m, k, rho, p, u, ph->penalty, st, &sc32)) != DG_OK) return rc;
        Vmult A32 = make_vmult32(&sc32);
        rc = gmres_ir(m, A, A32, rhs, pnew, opts->gmres.rtol, opts->gmres.restart, opts->gmres.maxit,
                      opts->gmres.inner_rtol, &gi, st, pc);
      } else {
        rc = gmres(m, A, rhs, pnew, opts->gmres.rtol, opts->gmres.restart, opts->gmres.maxit, &gi, st, false,
                   pc);
      }
      if (rc != DG_OK && rc != DG_ERR_NOT_CONVERGED) return rc;
      inf.gmres_iters_total += gi.iters;
      inf.refinements_total += gi.refinements;
      if (gi.relres > inf.max_relres) inf.max_relres = gi.relres;
      if ((rc = recover_rt(m, k, rho, u, mhat, pnew, unew, st)) != DG_OK) return rc;
      DG_RUN(m, K_PICARD_NORMS, st, k_picard_norms<<<RED_BLOCKS, 256, 0, st>>>(p, pnew, u, unew, n, red.partial));
      DG_RUN(m, K_REDUCE, st, k_reduce_partials<<<4, 256, 0, st>>>(red.partial, 4, RED_BLOCKS, red.out));
      double s4[4];
      DG_CUDA(cudaMemcpyAsync(s4, red.out, sizeof(s4), cudaMemcpyDeviceToHost, st));
      DG_CUDA(cudaStreamSynchronize(st));
      std::swap(p, pnew);
      std::swap(u, unew);
      if (!std::isfinite(s4[0] + s4[1] + s4[2] + s4[3])) {
        set_error("imex_ark2_step: non-finite Picard iterate");
        return DG_ERR_NONFINITE;
      }
      const double dp = std::sqrt(s4[0] / (s4[1] > 0 ? s4[1] : 1e-300));
      const double du = s4[3] > 0 ? std::sqrt(s4[2] / s4[3]) : 0.0;
      if (opts->picard_fixed <= 0 && std::max(dp, du) < opts->picard_rtol) {
        ++kk;
        break;
      }
    }
    inf.picard_iters[l] = kk;
    if (m->gll) {
      if ((rc = stage_state_gll(m, rho, u, p, ph->gamma, y, st)) != DG_OK) return rc;
    } else {
      DG_RUN(m, K_STAGE, st, k_stage_state<<<gb, 256, 0, st>>>(rho, u, p, n, ph->gamma, y));
    }
    DG_LAUNCH_CHECK("stage state");
    if (incr) {
      rc = explicit_increment(m, pk, y, q, Fns[0], Fs[0], Fns[l], Fs[l], st);
      // Fns[0] already holds the damping at q: add its increment only
      if (rc == DG_OK) rc = sponge_rt(m, y, Fns[l], st, q);
    } else {
      rc = explicit_rt(m, ph, y, Fns[l], Fs[l], st);
    }
    if (rc != DG_OK) return rc;
    yprev = y;
    // the next stage reads y as its initial guess before overwriting it
  }
  StageCoefs fin{};
  fin.nst = 3;
  fin.dt = dt;
  for (int s = 0; s < 3; ++s) {
    fin.fns[s] = Fns[s];
    fin.fs[s] = Fs[s];
    fin.a[s] = bw[s];
  }
  DG_RUN(m, K_STAGE, st, k_final_update<<<gb, 256, 0, st>>>(q, n, fin, nullptr));
  DG_LAUNCH_CHECK("final update");
  DG_CUDA(cudaStreamSynchronize(st));
  if (info) *info = inf;
  return DG_OK;
}

__global__ void k_fill(double* __restrict__ a, int64_t n, double v) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

// Time the schedules of one precision and keep the fastest: the tile
// multiplier (cells per block) of the explicit operator's cell kernel
// (FP64), and the schedule of the fused Schur vmult (plus-side traces from
// a trace array or the neighbours' node lines, or one thread per x-line
// with its cells per block), timed over whole vmults.
static int tune_precision(dg_mesh* m, int prec, const double* q, const double* rho, const double* p,
                          const double* u, double* x, double* y, double* fns, double* fs, cudaStream_t st) {
  const bool fp32 = prec != DG_FP64 && prec != DG_PAIRS;
  dg_phys ph{1.4, 9.81, 1e-4, DG_R2, 1, prec, nullptr, 0.0};
  ImplK k = impl_consts(&ph, 1.0);
  int rc;
  if (prec == DG_FP64) {
    const int cand[3] = {1, 2, 4};
    double best = 1e300;
    int pick = 1;
    for (int c : cand) {
      m->tile[K_VOL_EXPLICIT] = c;
      for (int w = 0; w < 2; ++w)
        if ((rc = explicit_rt(m, &ph, q, fns, fs, st)) != DG_OK) return rc;
      m->prof.reset();
      m->prof.time_mask = 1u << K_VOL_EXPLICIT;
      m->prof.on = true;
      for (int rep = 0; rep < 4; ++rep)
        if ((rc = explicit_rt(m, &ph, q, fns, fs, st)) != DG_OK) return rc;
      dg_kernel_stat stats[K_COUNT];
      int nst = 0;
      if ((rc = dg_profile_end(m, stats, K_COUNT, &nst)) != DG_OK) return rc;
      const dg_kernel_stat& s = stats[K_VOL_EXPLICIT];
      if (s.timed_launches == 0) continue;
      const double t = s.total_ms / (double)s.timed_launches;
      if (t < best) {
        best = t;
        pick = c;
      }
    }
    m->tile[K_VOL_EXPLICIT] = pick;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  DG_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(cudaGetLastError(), "cudaEventCreate");
  }
  double best = 1e300;
  const int slot = prec == DG_FP64 ? 0 : (prec == DG_PAIRS ? 2 : 1);
  int* tiles = prec == DG_FP64 ? m->tile : (prec == DG_PAIRS ? m->tilep : m->tile32);
  int pick = m->fused_stage[slot], pick_tg = tiles[K_VOL_GRAD], pick_td = tiles[K_VOL_DIV];
  // candidates: trace array, neighbour node lines, and (3D, degree 3) one
  // thread per x-line with 1, 2 or 4 times the base cells per block
  struct Cand { int sched, tile; };
  Cand cand[5] = {{0, 1}, {1, 1}, {2, 1}, {2, 2}, {2, 4}};
  const int ncand = (m->dim == 3 && m->n == 4 && m->terrain) ? 5 : 2;   // where schedule 2 runs
  rc = DG_OK;
  for (int ci = 0; ci < ncand && rc == DG_OK; ++ci) {
    const int sv = cand[ci].sched;
    m->fused_stage[slot] = sv;
    tiles[K_VOL_GRAD] = tiles[K_VOL_DIV] = cand[ci].tile;
    SchurCtx sc{m, k, rho, p, 1};
    Schur32Ctx sc32;
    SchurDfCtx sdf;
    Vmult A{nullptr, nullptr};
    if (prec == DG_PAIRS) {
      if ((rc = prepare_pairs(m, k, rho, p, u, 1, st, &sdf)) != DG_OK) break;
      A = make_vmult_pairs(&sdf);
    } else if (fp32) {
      if ((rc = prepare32(m, k, rho, p, u, 1, st, &sc32)) != DG_OK) break;
      A = make_vmult32(&sc32);
    } else {
      if ((rc = prepare_rt(m, k, rho, p, u, 1, st)) != DG_OK) break;
      A = make_vmult(&sc);
    }
    for (int w = 0; w < 2 && rc == DG_OK; ++w) rc = A(x, y, st);
    if (rc != DG_OK) break;
    cudaEventRecord(e0, st);
    for (int rep = 0; rep < 5 && rc == DG_OK; ++rep) rc = A(x, y, st);
    cudaEventRecord(e1, st);
    if (rc != DG_OK) break;
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "autotune timing");
      break;
    }
    if (ms < best) {
      best = ms;
      pick = sv;
      pick_tg = pick_td = cand[ci].tile;
    }
  }
  tiles[K_VOL_GRAD] = pick_tg;
  tiles[K_VOL_DIV] = pick_td;
  m->fused_stage[slot] = pick;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

}  // namespace dg

extern "C" int dg_mesh_autotune(dg_ctx* ctx, dg_mesh* m, int precision, void* stream) {
  if (!ctx || !m) {
    set_error("dg_mesh_autotune: NULL argument");
    return DG_ERR_ARG;
  }
  if (precision != DG_FP64 && precision != DG_MIXED && precision != DG_MIXED_EXPLICIT && precision != DG_PAIRS) {
    set_error("dg_mesh_autotune: precision must be DG_FP64, DG_MIXED, DG_MIXED_EXPLICIT or DG_PAIRS");
    return DG_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = m->N;
  double* buf = nullptr;
  // q (5n), rho, p, u (3n), x, y, fns (5n), fs (4n)
  DG_CUDA(cudaMalloc(&buf, sizeof(double) * 21 * n));
  double *q = buf, *rho = q + 5 * n, *p = rho + n, *u = p + n, *x = u + 3 * n, *y = x + n, *fns = y + n,
         *fs = fns + 5 * n;
  const unsigned gb = grid_for(n, 256);
  k_fill<<<gb, 256, 0, st>>>(q, n, 1.2);
  k_fill<<<gb, 256, 0, st>>>(q + n, n, 12.0);
  k_fill<<<gb, 256, 0, st>>>(q + 2 * n, 2 * n, 1.0);
  k_fill<<<gb, 256, 0, st>>>(q + 4 * n, n, 2.5e5);
  k_fill<<<gb, 256, 0, st>>>(rho, n, 1.2);
  k_fill<<<gb, 256, 0, st>>>(p, n, 1.0e5);
  k_fill<<<gb, 256, 0, st>>>(u, 3 * n, 10.0);
  k_fill<<<gb, 256, 0, st>>>(x, n, 1.0);
  int rc = cudaGetLastError() == cudaSuccess ? DG_OK : DG_ERR_CUDA;
  if (rc == DG_OK) rc = tune_precision(m, DG_FP64, q, rho, p, u, x, y, fns, fs, st);
  if (rc == DG_OK && precision != DG_FP64) rc = tune_precision(m, precision, q, rho, p, u, x, y, fns, fs, st);
  cudaStreamSynchronize(st);
  cudaFree(buf);
  return rc;
}
