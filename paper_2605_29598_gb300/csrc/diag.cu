// Diagnostics of a state: the geostrophic imbalance E_geo (Section 4,
// planetary-scale inertia-gravity wave, eq. egeo).
#include "solver.cuh"

namespace dg {

// per-block sums of (1 / invM) |F / rho| and (1 / invM): the volume integral
// of |F / rho| and the domain measure (w det J = 1 / invM at each node)
__global__ void k_geo_partials(const double* __restrict__ F, const double* __restrict__ rho,
                               const double* __restrict__ invM, int64_t n, double* __restrict__ partial) {
  __shared__ double red[2][256];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  double s0 = 0, s1 = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const double wj = 1.0 / invM[i];
    s0 += wj * fabs(F[i] / rho[i]);
    s1 += wj;
  }
  red[0][threadIdx.x] = s0;
  red[1][threadIdx.x] = s1;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[blockIdx.x * 2] = red[0][0];
    partial[blockIdx.x * 2 + 1] = red[1][0];
  }
}

}  // namespace dg

using namespace dg;

extern "C" int dg_geostrophic_error(dg_ctx* ctx, const dg_mesh* mesh, const dg_phys* ph, const double* q,
                                    double* e_geo, void* stream) {
  if (!ctx || !mesh || !ph || !q || !e_geo) {
    set_error("dg_geostrophic_error: NULL argument");
    return DG_ERR_ARG;
  }
  if (!(ph->gamma > 1.0)) {
    set_error("dg_geostrophic_error: gamma must be > 1");
    return DG_ERR_ARG;
  }
  if (mesh->gll) {
    set_error("dg_geostrophic_error: not implemented for Gauss-Lobatto nodes");
    return DG_ERR_UNSUPPORTED;
  }
  dg_mesh* m = const_cast<dg_mesh*>(mesh);
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = m->N;
  int rc;
  if ((rc = m->fns.ensure(sizeof(double) * 5 * n)) != DG_OK) return rc;
  if ((rc = m->fs.ensure(sizeof(double) * 4 * n)) != DG_OK) return rc;
  Red red;
  if ((rc = ensure_red(m, &red)) != DG_OK) return rc;
  double* fns = m->fns.as<double>();
  double* fs = m->fs.as<double>();
  // the scheme's own FP64 pressure gradient and Coriolis term: the stiff
  // x-momentum rate -dp/dx + f rho v
  PhysK k{ph->gamma, ph->g, ph->f, ph->f_cell, ph->lambda_min};
  rc = DG_ERR_UNSUPPORTED;
  DG_DISPATCH(m, rc = (Engine<double, D_, N_>::explicit_rates(m, k, q, fns, fs, st)));
  if (rc != DG_OK) return rc;
  DG_RUN(m, K_REDUCE, st, k_geo_partials<<<RED_BLOCKS, 256, 0, st>>>(fs, q, m->invM, n, red.partial));
  DG_RUN(m, K_REDUCE, st, k_reduce_partials<<<2, 256, 0, st>>>(red.partial, 2, RED_BLOCKS, red.out));
  DG_LAUNCH_CHECK("geostrophic error");
  double s[2];
  DG_CUDA(cudaMemcpyAsync(s, red.out, sizeof(s), cudaMemcpyDeviceToHost, st));
  DG_CUDA(cudaStreamSynchronize(st));
  if (!std::isfinite(s[0])) {
    set_error("dg_geostrophic_error: non-finite value");
    return DG_ERR_NONFINITE;
  }
  *e_geo = s[0] / s[1];
  return DG_OK;
}
