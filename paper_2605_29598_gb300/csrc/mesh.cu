// Context, error plumbing, 1D tables and mesh creation (validation, face
// lists, geometry) of libdgimex.
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace dg {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
}

int DBuf::ensure(size_t nbytes) {
  if (nbytes <= bytes && p) return DG_OK;
  release();
  cudaError_t e = cudaMalloc(&p, nbytes ? nbytes : 16);
  if (e != cudaSuccess) {
    p = nullptr;
    bytes = 0;
    return cuda_fail(e, "cudaMalloc(workspace)");
  }
  bytes = nbytes;
  return DG_OK;
}

void DBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

const char* const kKernelNames[K_COUNT] = {
    "trace", "face_explicit", "hang_gather", "volume_explicit", "face_lambda", "face_grad",
    "volume_grad", "face_div", "volume_div", "ustar", "multidot", "reduce", "multiaxpy", "vector",
    "stage", "picard_norms", "precond", "precond_setup"};

cudaEvent_t Profiler::next_event() {
  if (used == pool.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    pool.push_back(e);
  }
  return pool[used++];
}

void Profiler::reset() {
  for (int k = 0; k < K_COUNT; ++k) launches[k] = 0;
  used = 0;
  pending_kid.clear();
}

void Profiler::release() {
  for (auto e : pool) cudaEventDestroy(e);
  pool.clear();
  reset();
}

// Gauss-Legendre nodes on [-1, 1] by Newton iteration on P_n (three-term
// recurrence), mapped to [0, 1]; Lagrange values and derivatives by the
// product rule.
void make_tables(int n, HostTables* out) {
  out->n = n;
  for (int i = 0; i < n; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double pn = n == 0 ? 1.0 : (n == 1 ? t : p1);
      double pm = n == 1 ? 1.0 : p0;
      dp = n * (t * pn - pm) / (t * t - 1.0);
      double dt = pn / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    // node i counted from the right end; store ascending
    out->x[n - 1 - i] = 0.5 * (t + 1.0);
    out->w[n - 1 - i] = 1.0 / ((1.0 - t * t) * dp * dp);   // 2/((1-t^2)P'^2) / 2
  }
  const double* x = out->x;
  auto lag = [&](int j, double s) {
    double v = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) v *= (s - x[k]) / (x[j] - x[k]);
    return v;
  };
  auto dlag = [&](int j, double s) {
    double acc = 0.0;
    for (int m = 0; m < n; ++m) {
      if (m == j) continue;
      double v = 1.0 / (x[j] - x[m]);
      for (int k = 0; k < n; ++k)
        if (k != j && k != m) v *= (s - x[k]) / (x[j] - x[k]);
      acc += v;
    }
    return acc;
  };
  std::memset(&out->t, 0, sizeof(out->t));
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j) {
      out->t.D[k][j] = dlag(j, x[k]);
      out->t.P[0][k][j] = lag(j, 0.5 * x[k]);
      out->t.P[1][k][j] = lag(j, 0.5 * (x[k] + 1.0));
    }
  for (int j = 0; j < n; ++j) {
    out->t.L[0][j] = lag(j, 0.0);
    out->t.L[1][j] = lag(j, 1.0);
  }
  // Gauss-Lobatto nodes: the ends and the roots of P'_{n-1} on [-1, 1],
  // in closed form for n <= 5
  static const double gll_in[MAX_N + 1][MAX_N] = {
      {0}, {0.0}, {-1.0, 1.0}, {-1.0, 0.0, 1.0},
      {-1.0, -0.44721359549995793928, 0.44721359549995793928, 1.0},   // +-1/sqrt 5
      {-1.0, -0.65465367070797714380, 0.0, 0.65465367070797714380, 1.0}};   // +-sqrt(3/7)
  double* xl = out->xl;
  for (int k = 0; k < n; ++k) xl[k] = 0.5 * (gll_in[n][k] + 1.0);
  auto lagl = [&](int j, double s) {
    double v = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) v *= (s - xl[k]) / (xl[j] - xl[k]);
    return v;
  };
  std::memset(&out->G, 0, sizeof(out->G));
  std::memset(&out->Gi, 0, sizeof(out->Gi));
  for (int q = 0; q < n; ++q)
    for (int j = 0; j < n; ++j) {
      out->G.m[q][j] = lagl(j, x[q]);
      out->Gi.m[q][j] = lag(j, xl[q]);
    }
}

// ---------------------------------------------------------------------------
// geometry kernels
// ---------------------------------------------------------------------------

struct GeoArgs {
  const double* verts;
  int dim, n, Np, nfp;
  int64_t E;
  double x[MAX_N], w[MAX_N];
};

// Jacobian columns t_c = dx/dxi_c of the multilinear map at reference point xi.
__device__ void jac(const double* V, int dim, const double* xi, double J[3][3]) {
  for (int b = 0; b < 3; ++b)
    for (int c = 0; c < 3; ++c) J[b][c] = 0.0;
  int nv = 1 << dim;
  for (int v = 0; v < nv; ++v) {
    for (int c = 0; c < dim; ++c) {
      double wgt = 1.0;
      for (int a = 0; a < dim; ++a) {
        int bit = (v >> a) & 1;
        if (a == c) wgt *= bit ? 1.0 : -1.0;
        else wgt *= bit ? xi[a] : 1.0 - xi[a];
      }
      for (int b = 0; b < dim; ++b) J[b][c] += wgt * V[v * dim + b];
    }
  }
}

// adj[a][b] = det(J) * (J^{-1})[a][b]
__device__ double adjugate(int dim, const double J[3][3], double adj[3][3]) {
  if (dim == 2) {
    adj[0][0] = J[1][1];
    adj[0][1] = -J[0][1];
    adj[1][0] = -J[1][0];
    adj[1][1] = J[0][0];
    return J[0][0] * J[1][1] - J[0][1] * J[1][0];
  }
  // rows of adj are cross products of the Jacobian columns
  for (int a = 0; a < 3; ++a) {
    int c1 = (a + 1) % 3, c2 = (a + 2) % 3;
    adj[a][0] = J[1][c1] * J[2][c2] - J[2][c1] * J[1][c2];
    adj[a][1] = J[2][c1] * J[0][c2] - J[0][c1] * J[2][c2];
    adj[a][2] = J[0][c1] * J[1][c2] - J[1][c1] * J[0][c2];
  }
  return J[0][0] * adj[0][0] + J[1][0] * adj[0][1] + J[2][0] * adj[0][2];
}

__global__ void k_volume_geometry(GeoArgs g, double* K, double* invM, int* bad) {
  int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t N = g.E * g.Np;
  if (node >= N) return;
  int64_t e = node / g.Np;
  int i = (int)(node % g.Np);
  double xi[3] = {0, 0, 0};
  double w = 1.0;
  for (int a = 0, r = i; a < g.dim; ++a, r /= g.n) {
    xi[a] = g.x[r % g.n];
    w *= g.w[r % g.n];
  }
  double J[3][3], adj[3][3];
  jac(g.verts + e * (int64_t)(g.dim << g.dim), g.dim, xi, J);
  double det = adjugate(g.dim, J, adj);
  if (!(det > 0.0)) atomicExch(bad, 1);
  for (int a = 0; a < g.dim; ++a)
    for (int b = 0; b < g.dim; ++b) K[(int64_t)(a * g.dim + b) * N + node] = w * adj[a][b];
  invM[node] = 1.0 / (w * det);
}

// n dS at each face point of the minus side (Nanson: det(J) J^{-T} e_a).
__global__ void k_face_geometry(GeoArgs g, const int* fp_minus, int64_t nF, double* fgeo) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= nF) return;
  int slot = fp_minus[p];
  int nfaces = 2 * g.dim;
  int pt = slot % g.nfp;
  int f = (slot / g.nfp) % nfaces;
  int64_t e = slot / (g.nfp * nfaces);
  int a = f / 2, s = f % 2;
  double xi[3] = {0, 0, 0};
  double w = 1.0;
  xi[a] = (double)s;
  for (int t = 0, r = pt; t < g.dim; ++t) {
    if (t == a) continue;
    xi[t] = g.x[r % g.n];
    w *= g.w[r % g.n];
    r /= g.n;
  }
  double J[3][3], adj[3][3];
  jac(g.verts + e * (int64_t)(g.dim << g.dim), g.dim, xi, J);
  adjugate(g.dim, J, adj);
  double sg = s ? 1.0 : -1.0, nn = 0.0;
  for (int b = 0; b < g.dim; ++b) {
    double v = sg * w * adj[a][b];
    fgeo[(int64_t)b * nF + p] = v;
    nn += v * v;
  }
  fgeo[(int64_t)g.dim * nF + p] = sqrt(nn);
}

__global__ void k_node_coords(GeoArgs g, double* xyz) {
  int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t N = g.E * g.Np;
  if (node >= N) return;
  int64_t e = node / g.Np;
  int i = (int)(node % g.Np);
  double xi[3] = {0, 0, 0};
  for (int a = 0, r = i; a < g.dim; ++a, r /= g.n) xi[a] = g.x[r % g.n];
  const double* V = g.verts + e * (int64_t)(g.dim << g.dim);
  for (int b = 0; b < g.dim; ++b) {
    double acc = 0.0;
    for (int v = 0; v < (1 << g.dim); ++v) {
      double wgt = 1.0;
      for (int a = 0; a < g.dim; ++a) wgt *= ((v >> a) & 1) ? xi[a] : 1.0 - xi[a];
      acc += wgt * V[v * g.dim + b];
    }
    xyz[(int64_t)b * N + node] = acc;
  }
}

__global__ void k_cast_f64_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// FP32 copies of the geometry for the FP32 operator kernels (made once).
int ensure_fp32_geometry(dg_mesh* m) {
  if (m->K32) return DG_OK;
  const int64_t nK = (int64_t)m->dim * m->dim * m->N, nG = (int64_t)(m->dim + 1) * (m->nF > 0 ? m->nF : 1);
  float *K32 = nullptr, *iM32 = nullptr, *g32 = nullptr;
  cudaError_t e = cudaMalloc(&K32, sizeof(float) * nK);
  if (e == cudaSuccess) e = cudaMalloc(&iM32, sizeof(float) * m->N);
  if (e == cudaSuccess) e = cudaMalloc(&g32, sizeof(float) * nG);
  if (e != cudaSuccess) {
    cudaFree(K32);
    cudaFree(iM32);
    cudaFree(g32);
    return cuda_fail(e, "cudaMalloc(fp32 geometry)");
  }
  k_cast_f64_f32<<<grid_for(nK, 256), 256>>>(m->K, K32, nK);
  k_cast_f64_f32<<<grid_for(m->N, 256), 256>>>(m->invM, iM32, m->N);
  if (m->nF > 0) k_cast_f64_f32<<<grid_for(nG, 256), 256>>>(m->fgeo, g32, nG);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaFree(K32);
    cudaFree(iM32);
    cudaFree(g32);
    return cuda_fail(e, "fp32 geometry");
  }
  m->K32 = K32;
  m->invM32 = iM32;
  m->fgeo32 = g32;
  // corner offsets relative to corner 0, formed in FP64 and rounded: the
  // FP32 metric built from them keeps FP32 relative accuracy however far the
  // cell is from the origin
  const int nv = m->dim << m->dim;
  std::vector<double> hv((size_t)m->E * nv);
  std::vector<float> lv((size_t)m->E * nv);
  e = cudaMemcpy(hv.data(), m->verts, sizeof(double) * hv.size(), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "fp32 corner offsets");
  for (int64_t c = 0; c < m->E; ++c)
    for (int v = 0; v < (1 << m->dim); ++v)
      for (int b = 0; b < m->dim; ++b)
        lv[c * nv + v * m->dim + b] = (float)(hv[c * nv + v * m->dim + b] - hv[c * nv + b]);
  float* lv32 = nullptr;
  e = cudaMalloc(&lv32, sizeof(float) * lv.size());
  if (e == cudaSuccess) e = cudaMemcpy(lv32, lv.data(), sizeof(float) * lv.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(lv32);
    return cuda_fail(e, "fp32 corner offsets");
  }
  m->lv32 = lv32;
  if (m->terrain) {
    // per cell: dx, dy, then the bilinear coefficients (a, b, c, d) of
    // dz/dxi_0 in (xi_1, xi_2), dz/dxi_1 in (xi_0, xi_2) and dz/dxi_2 in
    // (xi_0, xi_1) (3D; in 2D dz/dxi_0 = a0 + b0 xi_1, dz/dxi_1 = a1 + b1 xi_0),
    // all from the corner offsets in FP64
    const int d = m->dim;
    std::vector<float> tc((size_t)m->E * 16, 0.0f);
    for (int64_t c = 0; c < m->E; ++c) {
      const double* V = hv.data() + c * nv;
      auto z = [&](int v) { return V[v * d + d - 1] - V[d - 1]; };
      float* o = tc.data() + c * 16;
      o[0] = (float)(V[1 * d + 0] - V[0]);
      if (d == 3) {
        o[1] = (float)(V[2 * d + 1] - V[1]);
        double D[3][4];
        for (int j = 0; j < 4; ++j) {
          D[0][j] = z(2 * j + 1) - z(2 * j);                                   // bit 0 pairs, j = (b1, b2)
          const int v1 = (j & 1) | 2 | ((j >> 1) << 2);
          D[1][j] = z(v1) - z(v1 - 2);                                         // bit 1 pairs, j = (b0, b2)
          D[2][j] = z(j + 4) - z(j);                                           // bit 2 pairs, j = (b0, b1)
        }
        for (int r = 0; r < 3; ++r) {
          o[2 + 4 * r] = (float)D[r][0];
          o[3 + 4 * r] = (float)(D[r][1] - D[r][0]);
          o[4 + 4 * r] = (float)(D[r][2] - D[r][0]);
          o[5 + 4 * r] = (float)(D[r][3] - D[r][2] - D[r][1] + D[r][0]);
        }
      } else {
        o[2] = (float)(z(1) - z(0));
        o[3] = (float)((z(3) - z(2)) - (z(1) - z(0)));
        o[6] = (float)(z(2) - z(0));
        o[7] = (float)((z(3) - z(1)) - (z(2) - z(0)));
      }
    }
    float* tc32 = nullptr;
    e = cudaMalloc(&tc32, sizeof(float) * tc.size());
    if (e == cudaSuccess) e = cudaMemcpy(tc32, tc.data(), sizeof(float) * tc.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(tc32);
      return cuda_fail(e, "fp32 terrain coefficients");
    }
    m->tc32 = tc32;
  }
  return DG_OK;
}

// outward n dS of every face slot of its own cell (all S slots, including
// the coarse sides of 2:1 faces, which the face-point list does not hold)
__global__ void k_slot_normals(GeoArgs g, int64_t S, double* out) {
  const int64_t slot = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (slot >= S) return;
  const int nfaces = 2 * g.dim;
  const int pt = (int)(slot % g.nfp);
  const int f = (int)((slot / g.nfp) % nfaces);
  const int64_t e = slot / ((int64_t)g.nfp * nfaces);
  const int a = f / 2, s = f % 2;
  double xi[3] = {0, 0, 0};
  double w = 1.0;
  xi[a] = (double)s;
  for (int t = 0, r = pt; t < g.dim; ++t) {
    if (t == a) continue;
    xi[t] = g.x[r % g.n];
    w *= g.w[r % g.n];
    r /= g.n;
  }
  double J[3][3], adj[3][3];
  jac(g.verts + e * (int64_t)(g.dim << g.dim), g.dim, xi, J);
  adjugate(g.dim, J, adj);
  const double sg = s ? 1.0 : -1.0;
  for (int b = 0; b < g.dim; ++b) out[(int64_t)b * S + slot] = sg * w * adj[a][b];
}

static GeoArgs geo_args(const dg_mesh* m) {
  GeoArgs g;
  g.verts = m->verts;
  g.dim = m->dim;
  g.n = m->n;
  g.Np = m->Np;
  g.nfp = m->nfp;
  g.E = m->E;
  for (int k = 0; k < MAX_N; ++k) {
    g.x[k] = m->tab.x[k];
    g.w[k] = m->tab.w[k];
  }
  return g;
}

}  // namespace dg

using namespace dg;

int64_t dg_mesh::workspace_bytes() const {
  const DBuf* b[kBufs];
  bufs(b);
  int64_t s = 0;
  if (K32) s += (int64_t)sizeof(float) * ((int64_t)dim * dim * N + N + (int64_t)(dim + 1) * (nF > 0 ? nF : 1));
  for (auto* x : b) s += (int64_t)x->bytes;
  return s;
}

extern "C" {

const char* dg_status_string(int s) {
  switch (s) {
    case DG_OK: return "DG_OK";
    case DG_ERR_ARG: return "DG_ERR_ARG";
    case DG_ERR_UNSUPPORTED: return "DG_ERR_UNSUPPORTED";
    case DG_ERR_CUDA: return "DG_ERR_CUDA";
    case DG_ERR_NOT_CONVERGED: return "DG_ERR_NOT_CONVERGED";
    case DG_ERR_TIMEOUT: return "DG_ERR_TIMEOUT";
    case DG_ERR_NONFINITE: return "DG_ERR_NONFINITE";
    case DG_ERR_OOM: return "DG_ERR_OOM";
    default: return "DG_UNKNOWN";
  }
}

const char* dg_last_error(void) { return g_err; }

int dg_ctx_create(int device, dg_ctx** out) {
  if (!out) {
    set_error("dg_ctx_create: out is NULL");
    return DG_ERR_ARG;
  }
  int count = 0;
  DG_CUDA(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count) {
    set_error("dg_ctx_create: device %d not in [0, %d)", device, count);
    return DG_ERR_ARG;
  }
  DG_CUDA(cudaSetDevice(device));
  dg_ctx* c = new dg_ctx;
  c->device = device;
  *out = c;
  return DG_OK;
}

void dg_ctx_destroy(dg_ctx* ctx) { delete ctx; }

void dg_mesh_destroy(dg_mesh* m) {
  if (!m) return;
  cudaFree(m->verts);
  cudaFree(m->K);
  cudaFree(m->invM);
  cudaFree(m->fgeo);
  cudaFree(m->fp_minus);
  cudaFree(m->fp_plus);
  cudaFree(m->hp_cslot);
  cudaFree(m->hp_code);
  cudaFree(m->hc_slot);
  cudaFree(m->K32);
  cudaFree(m->invM32);
  cudaFree(m->fgeo32);
  cudaFree(m->lv32);
  cudaFree(m->tc32);
  cudaFree(m->vl_above);
  cudaFree(m->vl_below);
  cudaFree(m->vl_heads);
  cudaFree(m->cface);
  cudaFree(m->fp_far);
  cudaFree(m->far_p);
  graph_release(m);
  const DBuf* b[dg_mesh::kBufs];
  m->bufs(b);
  for (auto* x : b) const_cast<DBuf*>(x)->release();
  m->prof.release();
  delete m;
}

namespace {

// Hanging rows grouped by coarse face, in the order validation meets them.
struct HangGroups {
  std::vector<int64_t> list;   // coarse face keys e * 2d + f
  std::vector<int64_t> rows;   // 2^(dim-1) hang_faces rows per coarse face, by subface
};

// Every rule dg_mesh_create checks before its first CUDA call; `who` names
// the entry point in the error message.
int check_desc(const dg_mesh_desc* d, const char* who, HangGroups* hg) {
  if (d->dim != 2 && d->dim != 3) {
    set_error("%s: dim %d not in {2, 3}", who, d->dim);
    return DG_ERR_ARG;
  }
  if (d->degree < 1 || d->degree > 4) {
    set_error("%s: degree %d not in 1..4", who, d->degree);
    return d->degree > 4 ? DG_ERR_UNSUPPORTED : DG_ERR_ARG;
  }
  if (d->node_set != DG_NODES_GL && d->node_set != DG_NODES_GLL) {
    set_error("%s: unknown node_set %d", who, d->node_set);
    return DG_ERR_ARG;
  }
  if (d->n_elem <= 0 || !d->vertices || d->n_int < 0 || d->n_hang < 0 || d->n_bdry < 0 ||
      (d->n_int && !d->int_faces) || (d->n_hang && !d->hang_faces) ||
      (d->n_bdry && !d->bdry_faces)) {
    set_error("%s: empty mesh or NULL list", who);
    return DG_ERR_ARG;
  }
  const int dim = d->dim, n = d->degree + 1, nfaces = 2 * dim;
  const int nfp = ipow(n, dim - 1), nsub = 1 << (dim - 1);
  const int64_t E = d->n_elem;
  if (E * nfaces * (int64_t)nfp >= (int64_t)1 << 31 || E * ipow(n, dim) >= (int64_t)1 << 31) {
    set_error("%s: mesh too large for 32-bit slot indices", who);
    return DG_ERR_UNSUPPORTED;
  }
  // ---- validation: every cell face covered exactly once
  std::vector<uint8_t> cover((size_t)E * nfaces, 0);
  auto bad = [&](const char* what, int64_t row) {
    set_error("%s: %s (row %lld)", who, what, (long long)row);
    return DG_ERR_ARG;
  };
  for (int64_t k = 0; k < d->n_int; ++k) {
    const int64_t* r = d->int_faces + 4 * k;
    if (r[0] < 0 || r[0] >= E || r[2] < 0 || r[2] >= E) return bad("interior face cell out of range", k);
    if (r[1] < 0 || r[1] >= nfaces || r[3] < 0 || r[3] >= nfaces) return bad("interior face index out of range", k);
    if (r[1] % 2 != 1 || r[3] != r[1] - 1) return bad("interior face needs fL = 2a+1, fR = 2a", k);
    if (r[0] == r[2]) return bad("interior face joins a cell to itself", k);
    cover[r[0] * nfaces + r[1]]++;
    cover[r[2] * nfaces + r[3]]++;
  }
  for (int64_t k = 0; k < d->n_bdry; ++k) {
    const int64_t* r = d->bdry_faces + 3 * k;
    if (r[0] < 0 || r[0] >= E || r[1] < 0 || r[1] >= nfaces) return bad("boundary face out of range", k);
    if (r[2] != DG_BC_WALL && r[2] != DG_BC_FARFIELD) return bad("unknown boundary condition", k);
    cover[r[0] * nfaces + r[1]]++;
  }
  // group hanging rows by coarse face
  std::vector<int64_t> hc_first((size_t)E * nfaces, -1);
  std::vector<int64_t>& hc_list = hg->list;
  std::vector<int64_t>& hc_rows = hg->rows;
  for (int64_t k = 0; k < d->n_hang; ++k) {
    const int64_t* r = d->hang_faces + 5 * k;
    if (r[0] < 0 || r[0] >= E || r[2] < 0 || r[2] >= E) return bad("hanging face cell out of range", k);
    if (r[1] < 0 || r[1] >= nfaces || r[3] < 0 || r[3] >= nfaces) return bad("hanging face index out of range", k);
    if (r[3] != (r[1] ^ 1)) return bad("hanging face needs f_fine = f_coarse ^ 1", k);
    if (r[4] < 0 || r[4] >= nsub) return bad("subface index out of range", k);
    if (r[0] == r[2]) return bad("hanging face joins a cell to itself", k);
    cover[r[2] * nfaces + r[3]]++;
    int64_t key = r[0] * nfaces + r[1];
    if (hc_first[key] < 0) {
      hc_first[key] = (int64_t)hc_list.size();
      hc_list.push_back(key);
      hc_rows.insert(hc_rows.end(), nsub, -1);
      cover[key]++;
    }
    int64_t& slotrow = hc_rows[hc_first[key] * nsub + r[4]];
    if (slotrow >= 0) return bad("subface listed twice", k);
    slotrow = k;
  }
  for (size_t k = 0; k < hc_rows.size(); ++k)
    if (hc_rows[k] < 0) {
      set_error("%s: coarse face %lld misses a subface", who, (long long)(k / nsub));
      return DG_ERR_ARG;
    }
  for (int64_t k = 0; k < E * nfaces; ++k)
    if (cover[k] != 1) {
      set_error("%s: face %d of cell %lld covered %d times", who, (int)(k % nfaces),
                (long long)(k / nfaces), (int)cover[k]);
      return DG_ERR_ARG;
    }
  for (int64_t k = 0; k < E * (dim << dim); ++k)
    if (!std::isfinite(d->vertices[k])) return bad("non-finite vertex coordinate", k / (dim << dim));
  return DG_OK;
}

}  // namespace

int dg_mesh_create(dg_ctx* ctx, const dg_mesh_desc* d, dg_mesh** out) {
  if (!ctx || !d || !out) {
    set_error("dg_mesh_create: NULL argument");
    return DG_ERR_ARG;
  }
  *out = nullptr;
  HangGroups hg;
  {
    const int rc = check_desc(d, "dg_mesh_create", &hg);
    if (rc != DG_OK) return rc;
  }
  const int dim = d->dim, n = d->degree + 1, nfaces = 2 * dim;
  const int nfp = ipow(n, dim - 1), nsub = 1 << (dim - 1);
  const int64_t E = d->n_elem;
  const std::vector<int64_t>& hc_list = hg.list;
  const std::vector<int64_t>& hc_rows = hg.rows;

  // ---- unified face-point list
  const int64_t nHC = (int64_t)hc_list.size();
  const int64_t nH = nHC * nsub * nfp;
  const int64_t nF = (d->n_int + d->n_bdry) * nfp + nH;
  std::vector<int> fpm(nF), fpp(nF), hpc(nH), hpcode(nH), hcs(nHC);
  int64_t p = 0;
  for (int64_t k = 0; k < d->n_int; ++k) {
    const int64_t* r = d->int_faces + 4 * k;
    for (int t = 0; t < nfp; ++t, ++p) {
      fpm[p] = (int)((r[0] * nfaces + r[1]) * nfp + t);
      fpp[p] = (int)((r[2] * nfaces + r[3]) * nfp + t);
    }
  }
  for (int64_t k = 0; k < d->n_bdry; ++k) {
    const int64_t* r = d->bdry_faces + 3 * k;
    for (int t = 0; t < nfp; ++t, ++p) {
      fpm[p] = (int)((r[0] * nfaces + r[1]) * nfp + t);
      fpp[p] = -1;
    }
  }
  for (int64_t c = 0; c < nHC; ++c) {
    hcs[c] = (int)(hc_list[c] * nfp);
    for (int s = 0; s < nsub; ++s) {
      const int64_t* r = d->hang_faces + 5 * hc_rows[c * nsub + s];
      for (int t = 0; t < nfp; ++t, ++p) {
        int64_t hp = (c * nsub + s) * nfp + t;
        fpm[p] = (int)((r[2] * nfaces + r[3]) * nfp + t);
        fpp[p] = (int)(-2 - hp);
        hpc[hp] = hcs[c];
        hpcode[hp] = s | (t << 8);
      }
    }
  }

  // ---- vertical chains: cells linked through conforming top (2a+1) /
  // bottom (2a) faces of the last reference direction a = dim - 1; a
  // vertically periodic column is cut at its first cell
  std::vector<int> above((size_t)E, -1), below((size_t)E, -1), heads;
  for (int64_t k = 0; k < d->n_int; ++k) {
    const int64_t* r = d->int_faces + 4 * k;
    if (r[1] == 2 * (dim - 1) + 1) {
      above[r[0]] = (int)r[2];
      below[r[2]] = (int)r[0];
    }
  }
  {
    std::vector<uint8_t> seen((size_t)E, 0);
    auto walk = [&](int64_t c) {
      for (int64_t e = c; e >= 0 && !seen[e]; e = above[e]) seen[e] = 1;
    };
    for (int64_t c = 0; c < E; ++c)
      if (below[c] < 0) {
        heads.push_back((int)c);
        walk(c);
      }
    for (int64_t c = 0; c < E; ++c)
      if (!seen[c]) {
        above[below[c]] = -1;
        below[c] = -1;
        heads.push_back((int)c);
        walk(c);
      }
  }

  dg_mesh* m = new dg_mesh;
  m->ctx = ctx;
  m->dim = dim;
  m->degree = d->degree;
  m->n = n;
  m->Np = ipow(n, dim);
  m->nfp = nfp;
  m->nfaces = nfaces;
  m->E = E;
  m->N = E * m->Np;
  m->S = E * nfaces * nfp;
  m->nF = nF;
  m->nH = nH;
  m->nHC = nHC;
  m->gll = d->node_set == DG_NODES_GLL;
  make_tables(n, &m->tab);
  auto fail = [&](int st) {
    dg_mesh_destroy(m);
    return st;
  };
#define ALLOC(ptr, count)                                                      \
  do {                                                                         \
    cudaError_t e_ = cudaMalloc(&(ptr), sizeof(*(ptr)) * (size_t)((count) > 0 ? (count) : 1)); \
    if (e_ != cudaSuccess) return fail(cuda_fail(e_, "cudaMalloc(mesh)"));     \
  } while (0)
#define UPLOAD(dst, src, count)                                                \
  do {                                                                         \
    if ((count) > 0) {                                                         \
      cudaError_t e_ = cudaMemcpy(dst, src, sizeof(*(dst)) * (size_t)(count),  \
                                  cudaMemcpyHostToDevice);                     \
      if (e_ != cudaSuccess) return fail(cuda_fail(e_, "cudaMemcpy(mesh)"));   \
    }                                                                          \
  } while (0)
  ALLOC(m->verts, E * (dim << dim));
  ALLOC(m->K, (int64_t)dim * dim * m->N);
  ALLOC(m->invM, m->N);
  ALLOC(m->fgeo, (int64_t)(dim + 1) * nF);
  ALLOC(m->fp_minus, nF);
  ALLOC(m->fp_plus, nF);
  ALLOC(m->hp_cslot, nH);
  ALLOC(m->hp_code, nH);
  ALLOC(m->hc_slot, nHC);
  UPLOAD(m->verts, d->vertices, E * (dim << dim));
  {
    // terrain-following test: horizontal coordinate c of every corner equals
    // that of the corner with only bit c kept (exact comparison)
    bool tf = true;
    const int nc = 1 << dim;
    for (int64_t e = 0; e < E && tf; ++e) {
      const double* v = d->vertices + e * nc * dim;
      for (int c = 0; c < dim - 1 && tf; ++c)
        for (int k = 0; k < nc && tf; ++k)
          if (v[k * dim + c] != v[(k & (1 << c)) * dim + c]) tf = false;
    }
    m->terrain = tf;
  }
  UPLOAD(m->fp_minus, fpm.data(), nF);
  UPLOAD(m->fp_plus, fpp.data(), nF);
  UPLOAD(m->hp_cslot, hpc.data(), nH);
  UPLOAD(m->hp_code, hpcode.data(), nH);
  UPLOAD(m->hc_slot, hcs.data(), nHC);
  {
    // per-cell face codes of the fused face + cell kernels: the neighbour
    // cell across a conforming (or periodic) face, -1 on a wall, -2 on
    // either side of a 2:1 face
    std::vector<int> cf((size_t)E * nfaces, -1);
    for (int64_t k = 0; k < d->n_int; ++k) {
      const int64_t* r = d->int_faces + 4 * k;
      cf[r[0] * nfaces + r[1]] = (int)r[2];
      cf[r[2] * nfaces + r[3]] = (int)r[0];
    }
    for (int64_t k = 0; k < d->n_hang; ++k) {
      const int64_t* r = d->hang_faces + 5 * k;
      cf[r[0] * nfaces + r[1]] = -2;
      cf[r[2] * nfaces + r[3]] = -2;
    }
    // far-field faces: code -3, and the far-point list grouped by face type
    // (the boundary rows' face points follow the interior ones in the
    // unified list)
    std::vector<int> fpf((size_t)nF, -1), farp;
    const int64_t pb = d->n_int * nfp;
    for (int f = 0; f < nfaces; ++f) {
      m->far_fbeg[f] = (int64_t)farp.size();
      for (int64_t k = 0; k < d->n_bdry; ++k) {
        const int64_t* r = d->bdry_faces + 3 * k;
        if (r[2] != DG_BC_FARFIELD || r[1] != f) continue;
        cf[r[0] * nfaces + r[1]] = -3;
        for (int t = 0; t < nfp; ++t) {
          const int64_t p = pb + k * nfp + t;
          fpf[p] = (int)farp.size();
          farp.push_back((int)p);
        }
      }
    }
    m->far_fbeg[nfaces] = (int64_t)farp.size();
    m->nFar = (int64_t)farp.size();
    ALLOC(m->cface, E * nfaces);
    UPLOAD(m->cface, cf.data(), E * nfaces);
    if (m->nFar > 0) {
      ALLOC(m->fp_far, nF);
      ALLOC(m->far_p, m->nFar);
      UPLOAD(m->fp_far, fpf.data(), nF);
      UPLOAD(m->far_p, farp.data(), m->nFar);
    }
  }
  m->n_vchains = (int64_t)heads.size();
  ALLOC(m->vl_above, E);
  ALLOC(m->vl_below, E);
  ALLOC(m->vl_heads, m->n_vchains);
  UPLOAD(m->vl_above, above.data(), E);
  UPLOAD(m->vl_below, below.data(), E);
  UPLOAD(m->vl_heads, heads.data(), m->n_vchains);
#undef ALLOC
#undef UPLOAD
  GeoArgs g = geo_args(m);
  int* dbad = nullptr;
  {
    cudaError_t e = cudaMalloc(&dbad, sizeof(int));
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(flag)"));
  }
  cudaMemset(dbad, 0, sizeof(int));
  k_volume_geometry<<<grid_for(m->N, 256), 256>>>(g, m->K, m->invM, dbad);
  if (nF > 0) k_face_geometry<<<grid_for(nF, 256), 256>>>(g, m->fp_minus, nF, m->fgeo);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int hbad = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&hbad, dbad, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(dbad);
  if (e != cudaSuccess) return fail(cuda_fail(e, "mesh geometry"));
  if (hbad) {
    set_error("dg_mesh_create: a cell map has det(J) <= 0 at a node");
    return fail(DG_ERR_ARG);
  }
  *out = m;
  return DG_OK;
}

int dg_mesh_validate(const dg_mesh_desc* d) {
  if (!d) {
    set_error("dg_mesh_validate: NULL argument");
    return DG_ERR_ARG;
  }
  HangGroups hg;
  return check_desc(d, "dg_mesh_validate", &hg);
}

int dg_profile_begin(dg_mesh* m, uint32_t time_mask) {
  if (!m) {
    set_error("dg_profile_begin: NULL mesh");
    return DG_ERR_ARG;
  }
  m->prof.reset();
  m->prof.time_mask = time_mask;
  m->prof.on = true;
  return DG_OK;
}

int dg_profile_end(dg_mesh* m, dg_kernel_stat* out, int max_out, int* n_out) {
  if (!m || (max_out > 0 && !out)) {
    set_error("dg_profile_end: NULL argument");
    return DG_ERR_ARG;
  }
  Profiler& p = m->prof;
  p.on = false;
  double ms[K_COUNT] = {};
  int64_t timed[K_COUNT] = {};
  if (!p.pending_kid.empty()) DG_CUDA(cudaEventSynchronize(p.pool[2 * p.pending_kid.size() - 1]));
  for (size_t k = 0; k < p.pending_kid.size(); ++k) {
    float t = 0.f;
    DG_CUDA(cudaEventElapsedTime(&t, p.pool[2 * k], p.pool[2 * k + 1]));
    ms[p.pending_kid[k]] += t;
    timed[p.pending_kid[k]]++;
  }
  int n = max_out < K_COUNT ? max_out : K_COUNT;
  for (int k = 0; k < n; ++k) {
    std::memset(out[k].name, 0, sizeof(out[k].name));
    std::strncpy(out[k].name, kKernelNames[k], sizeof(out[k].name) - 1);
    out[k].launches = p.launches[k];
    out[k].timed_launches = timed[k];
    out[k].total_ms = ms[k];
  }
  if (n_out) *n_out = n;
  p.reset();
  return DG_OK;
}

int dg_mesh_info(const dg_mesh* m, dg_mesh_stats* o) {
  if (!m || !o) {
    set_error("dg_mesh_info: NULL argument");
    return DG_ERR_ARG;
  }
  o->dim = m->dim;
  o->degree = m->degree;
  o->n1d = m->n;
  o->nodes_per_elem = m->Np;
  o->n_elem = m->E;
  o->n_nodes = m->N;
  o->n_face_points = m->nF;
  o->n_hang_points = m->nH;
  o->workspace_bytes = m->workspace_bytes();
  const int kinds[3] = {K_VOL_EXPLICIT, K_VOL_GRAD, K_VOL_DIV};
  for (int k = 0; k < 3; ++k) {
    o->tile_fp64[k] = m->tile[kinds[k]];
    o->tile_fp32[k] = m->tile32[kinds[k]];
  }
  o->terrain_following = m->terrain ? 1 : 0;
  for (int k = 0; k < 3; ++k) o->fused_stage[k] = m->fused_stage[k];
  return DG_OK;
}

int dg_mesh_set_fused_stage(dg_mesh* m, int fp64, int fp32, int pairs) {
  if (!m || fp64 < 0 || fp64 > 2 || fp32 < 0 || fp32 > 2 || pairs < 0 || pairs > 2) {
    set_error("dg_mesh_set_fused_stage: mesh and 0, 1 or 2 per precision required");
    return DG_ERR_ARG;
  }
  m->fused_stage[0] = fp64;
  m->fused_stage[1] = fp32;
  m->fused_stage[2] = pairs;
  return DG_OK;
}

int dg_mesh_set_vmult_tile(dg_mesh* m, int precision, int tile) {
  if (!m || (tile != 1 && tile != 2 && tile != 4) ||
      (precision != DG_FP64 && precision != DG_MIXED && precision != DG_MIXED_EXPLICIT && precision != DG_PAIRS)) {
    set_error("dg_mesh_set_vmult_tile: mesh, a precision and a tile of 1, 2 or 4 required");
    return DG_ERR_ARG;
  }
  int* t = precision == DG_FP64 ? m->tile : (precision == DG_PAIRS ? m->tilep : m->tile32);
  t[dg::K_VOL_GRAD] = t[dg::K_VOL_DIV] = tile;
  return DG_OK;
}

}  // extern "C"

namespace dg {

int slot_normals(const dg_mesh* m, double* out, cudaStream_t st) {
  GeoArgs g = geo_args(m);
  if (m->S > 0) k_slot_normals<<<grid_for(m->S, 256), 256, 0, st>>>(g, m->S, out);
  DG_LAUNCH_CHECK("slot normals");
  return DG_OK;
}

}  // namespace dg

extern "C" {

int dg_mesh_node_coords(dg_ctx* ctx, const dg_mesh* m, double* xyz, void* stream) {
  if (!ctx || !m || !xyz) {
    set_error("dg_mesh_node_coords: NULL argument");
    return DG_ERR_ARG;
  }
  GeoArgs g = geo_args(m);
  if (m->gll)   // the nodes of a Gauss-Lobatto mesh
    for (int k = 0; k < MAX_N; ++k) g.x[k] = k < m->n ? m->tab.xl[k] : 0.0;
  k_node_coords<<<grid_for(m->N, 256), 256, 0, (cudaStream_t)stream>>>(g, xyz);
  DG_LAUNCH_CHECK("k_node_coords");
  return DG_OK;
}

}  // extern "C"
