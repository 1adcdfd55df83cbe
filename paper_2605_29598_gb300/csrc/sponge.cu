// Rayleigh damping (sponge) layers of the orography tests (Section 4, eq.
// damping): the non-stiff rates of every conserved field gain
// -lambda(x) (q - q_bar).  lambda is computed once per dg_mesh_set_sponge
// from the node coordinates; the damping itself is one pointwise pass after
// each evaluation of the explicit operator.
#include "solver.cuh"

namespace dg {

namespace {

__device__ __forceinline__ double sponge_ramp(double lam_bar, double t) {
  t = fmin(fmax(t, 0.0), 1.0);
  const double s = sin(0.5 * 3.14159265358979323846 * t);
  return lam_bar * s * s;
}

// lambda at every node: sin^2 ramps of the top layer and of the lateral
// layers towards both ends of x (and y in 3D); the largest applies
__global__ void k_sponge_lambda(const double* __restrict__ xyz, int dim, int64_t N, dg_sponge s,
                                double* __restrict__ lam) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double z = xyz[(int64_t)(dim - 1) * N + i];
  double l = z >= s.z_b ? sponge_ramp(s.lambda_bar, (z - s.z_b) / (s.z_t - s.z_b)) : 0.0;
  if (s.x_layers) {
    const double x = xyz[i];
    if (x <= s.x_lo + s.x_width) l = fmax(l, sponge_ramp(s.lambda_bar, (s.x_lo + s.x_width - x) / s.x_width));
    if (x >= s.x_hi - s.x_width) l = fmax(l, sponge_ramp(s.lambda_bar, (x - (s.x_hi - s.x_width)) / s.x_width));
  }
  if (s.y_layers && dim == 3) {
    const double y = xyz[N + i];
    if (y <= s.y_lo + s.y_width) l = fmax(l, sponge_ramp(s.lambda_bar, (s.y_lo + s.y_width - y) / s.y_width));
    if (y >= s.y_hi - s.y_width) l = fmax(l, sponge_ramp(s.lambda_bar, (y - (s.y_hi - s.y_width)) / s.y_width));
  }
  lam[i] = l;
}

// fns -= lambda (q - qbar) for the five fields of every damped node (qbar:
// the background, or the reference state of an increment)
__global__ void k_sponge(double* __restrict__ fns, const double* __restrict__ q, const double* __restrict__ lam,
                         const double* __restrict__ qbar, int64_t N) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double l = lam[i];
  if (l == 0.0) return;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int64_t j = (int64_t)k * N + i;
    fns[j] -= l * (q[j] - qbar[j]);
  }
}

}  // namespace

int sponge_rt(dg_mesh* m, const double* q, double* fns, cudaStream_t st, const double* ref) {
  if (!m->sponge_set) return DG_OK;
  const double* lam = m->sponge.as<double>();
  DG_RUN(m, K_STAGE, st, k_sponge<<<grid_for(m->N, 256), 256, 0, st>>>(fns, q, lam, ref ? ref : lam + m->N, m->N));
  DG_LAUNCH_CHECK("sponge");
  return DG_OK;
}

}  // namespace dg

using namespace dg;

extern "C" int dg_mesh_set_sponge(dg_ctx* ctx, dg_mesh* m, const dg_sponge* s, const double* q_bar, void* stream) {
  if (!ctx || !m) {
    set_error("dg_mesh_set_sponge: NULL argument");
    return DG_ERR_ARG;
  }
  if (!s) {
    m->sponge_set = false;
    return DG_OK;
  }
  if (m->gll) {
    set_error("dg_mesh_set_sponge: not implemented for Gauss-Lobatto nodes");
    return DG_ERR_UNSUPPORTED;
  }
  if (!q_bar || !(s->lambda_bar >= 0.0) || !(s->z_t > s->z_b) || (s->x_layers && !(s->x_width > 0.0)) ||
      (s->y_layers && !(s->y_width > 0.0))) {
    set_error("dg_mesh_set_sponge: q_bar required, lambda_bar >= 0, z_t > z_b, layer widths > 0");
    return DG_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t N = m->N;
  int rc;
  if ((rc = m->sponge.ensure(sizeof(double) * 6 * (size_t)N)) != DG_OK) return rc;
  double* lam = m->sponge.as<double>();
  double* qb = lam + N;
  // node coordinates go through the q_bar slot (dim x N <= 5 x N) first
  if ((rc = dg_mesh_node_coords(ctx, m, qb, stream)) != DG_OK) return rc;
  k_sponge_lambda<<<grid_for(N, 256), 256, 0, st>>>(qb, m->dim, N, *s, lam);
  DG_LAUNCH_CHECK("sponge coefficient");
  DG_CUDA(cudaMemcpyAsync(qb, q_bar, sizeof(double) * 5 * N, cudaMemcpyDeviceToDevice, st));
  m->sponge_set = true;
  return DG_OK;
}
