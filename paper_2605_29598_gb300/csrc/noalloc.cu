// Allocation-free variant of the explicit operator.
//
// dg_apply_explicit grows per-mesh device workspace with cudaMalloc the
// first time it runs on a mesh.  Some callers cannot allow that: a service
// that reserves all of its device memory up front and forbids allocation in
// its steady-state loop, or a host framework that owns every device
// allocation through its own pool and rejects raw cudaMalloc (which can
// also synchronise the device).  dg_apply_explicit_noalloc runs the same
// kernels with its scratch (face traces, face fluxes, 2:1 mortar values)
// taken from one fixed-size array of device memory that is part of the
// library image, so the call itself allocates nothing.
#include <mutex>

#include "engine.cuh"

namespace dg {

// Scratch capacity in doubles (32 MiB).  Every GPU that loads the library
// holds this array until the process exits.
constexpr int64_t NOALLOC_SCRATCH_DOUBLES = int64_t(1) << 22;

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

// Host code must not use g_noalloc_scratch directly: on the host that name
// is a stand-in object, not a device address.  The device address is
// looked up once per device and cached here.
constexpr int NOALLOC_MAX_DEVICES = 64;
static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

static int noalloc_scratch(int device, double** out) {
  if (device < 0 || device >= NOALLOC_MAX_DEVICES) {
    set_error("dg_apply_explicit_noalloc: device %d out of range", device);
    return DG_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_ptr[device] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[device];
  return DG_OK;
}

template <int DIM, int N>
static int explicit_with_scratch(dg_mesh* m, const PhysK& ph, const double* q, double* fns, double* fs,
                                 double* scratch, cudaStream_t st) {
  using CS = CellShape<DIM, N>;
  using T = double;
  Tables<T> tb = cast_tables<T>(m->tab.t);
  FaceTopo ft = topo(m);
  T* trc = scratch;                 // 5 x S
  T* slot = scratch + 5 * m->S;     // 9 x S
  T* hbuf = scratch + 14 * m->S;    // 9 x nH
  Fields<T> in;
  for (int k = 0; k < 5; ++k) {
    in.f[k] = q + k * m->N;
    in.scale[k] = 1;
  }
  DG_RUN(m, K_TRACE, st, k_trace<T, DIM, N, 5><<<trace_grid<DIM, N>(m->E), TraceShape<DIM, N>::THREADS, 0, st>>>(in, m->E, m->N, trc, m->S, tb));
  DG_RUN(m, K_FACE_EXPLICIT, st,
         k_face_explicit<T, DIM, N><<<grid_for(m->nF, 128), 128, 0, st>>>(ft, trc, slot, hbuf, tb, (T)ph.gamma,
                                                                       (T)ph.lambda_min));
  if (m->nHC > 0)
    DG_RUN(m, K_HANG_GATHER, st,
           k_hang_gather<T, DIM, N, 9><<<grid_for(m->nHC * CS::NFP, 128), 128, 0, st>>>(ft, hbuf, slot, tb));
  DG_TILE(m, K_VOL_EXPLICIT,
          DG_RUN(m, K_VOL_EXPLICIT, st,
                 k_volume_explicit<T, DIM, N, M_><<<grid_for(m->E, CellShape<DIM, N, M_>::EPB),
                                                    CellShape<DIM, N, M_>::THREADS, 0, st>>>(
                     q, m->K, m->invM, slot, m->E, m->S, tb, ph, fns, fs, m->terrain ? 1 : 0)));
  DG_LAUNCH_CHECK("explicit operator (no-alloc)");
  // damping layers: one pointwise pass over stored coefficients, no scratch
  return sponge_rt(m, q, fns, st);
}

}  // namespace dg

using namespace dg;

extern "C" int dg_apply_explicit_noalloc(dg_ctx* ctx, const dg_mesh* mesh, const dg_phys* ph, const double* q,
                                         double* fns, double* fs, void* stream) {
  if (!ctx || !mesh || !ph || !q || !fns || !fs) {
    set_error("dg_apply_explicit_noalloc: NULL argument");
    return DG_ERR_ARG;
  }
  if (!(ph->gamma > 1.0)) {
    set_error("dg_apply_explicit_noalloc: gamma must be > 1");
    return DG_ERR_ARG;
  }
  if (!(ph->lambda_min >= 0.0)) {
    set_error("dg_apply_explicit_noalloc: lambda_min must be >= 0");
    return DG_ERR_ARG;
  }
  if (mesh->gll) {
    set_error("dg_apply_explicit_noalloc: not implemented for Gauss-Lobatto nodes");
    return DG_ERR_UNSUPPORTED;
  }
  if (mesh->nFar > 0 && !mesh->far_set) {
    set_error("dg_apply_explicit_noalloc: set the far-field outer state with dg_mesh_set_far_state first");
    return DG_ERR_ARG;
  }
  if (ph->variant != DG_R1 && ph->variant != DG_R2) {
    set_error("dg_apply_explicit_noalloc: variant must be DG_R1 or DG_R2");
    return DG_ERR_ARG;
  }
  // DG_FP64 and DG_MIXED both evaluate the explicit operator in FP64 (as
  // dg_apply_explicit does); the FP32 perturbation form needs per-mesh
  // background buffers and is not offered here
  if (ph->precision == DG_MIXED_EXPLICIT) {
    set_error("dg_apply_explicit_noalloc: DG_MIXED_EXPLICIT is not implemented (use DG_FP64 or DG_MIXED)");
    return DG_ERR_UNSUPPORTED;
  }
  if (ph->precision != DG_FP64 && ph->precision != DG_MIXED) {
    set_error("dg_apply_explicit_noalloc: precision must be DG_FP64 or DG_MIXED");
    return DG_ERR_ARG;
  }
  const int64_t need = 14 * mesh->S + 9 * mesh->nH;
  if (need > NOALLOC_SCRATCH_DOUBLES) {
    set_error("dg_apply_explicit_noalloc: mesh needs %lld scratch doubles (14 per face point slot + 9 per "
              "hanging point), the fixed capacity is %lld; use dg_apply_explicit",
              (long long)need, (long long)NOALLOC_SCRATCH_DOUBLES);
    return DG_ERR_ARG;
  }
  int dev = -1;
  DG_CUDA(cudaGetDevice(&dev));
  if (dev != ctx->device) {
    set_error("dg_apply_explicit_noalloc: current device %d is not the context's device %d", dev, ctx->device);
    return DG_ERR_ARG;
  }
  double* scratch = nullptr;
  int rc = noalloc_scratch(dev, &scratch);
  if (rc != DG_OK) return rc;
  dg_mesh* m = const_cast<dg_mesh*>(mesh);
  PhysK k{ph->gamma, ph->g, ph->f, ph->f_cell, ph->lambda_min};
  DG_DISPATCH(m, return explicit_with_scratch<D_, N_>(m, k, q, fns, fs, scratch, (cudaStream_t)stream));
  set_error("dg_apply_explicit_noalloc: unsupported (dim, degree)");
  return DG_ERR_UNSUPPORTED;
}
