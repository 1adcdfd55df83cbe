// Device-driven ARK2 step: the whole step (Section 3: explicit rates, stage
// predictors, Picard loop around the Schur solve and the velocity recovery,
// final update) captured once as a CUDA graph and replayed.  The host-driven
// step reads every Arnoldi column back to run the Givens rotations and the
// stopping tests on the CPU; here those run in single-thread kernels and
// steer CUDA-graph "while" nodes (Picard loop, refinement sweeps, GMRES
// restart cycles, Arnoldi steps), so a step is one graph launch and one
// read-back of its counters.
//
// Every loop is bounded by a counter that its own check kernel increments:
// Arnoldi steps by the restart length, restart cycles and refinement sweeps
// by the iteration limit (sweeps also by 60), Picard iterations by
// picard_maxit.  Loop conditions are false on NaN.
#include <cstring>

#include "solver.cuh"

namespace dg {

constexpr int DSTRIDE = MAX_RESTART + 2;   // stride of the device-driven partial sums

// one restarted GMRES solve (device memory)
struct GmState {
  double H[(MAX_RESTART + 1) * MAX_RESTART];
  double cs[MAX_RESTART], sn[MAX_RESTART], g[MAX_RESTART + 1], y[MAX_RESTART];
  double c[MAX_RESTART + 2];     // Gram-Schmidt coefficients (-h)
  double dot[MAX_RESTART + 2];   // reduced dot products
  double bnorm, beta, tol, relres, w2, inv;
  int j, it, jused, maxit, restart, cycles, reorth, status;
};

// refinement sweeps of the mixed-precision solve
struct IrState {
  double dot0, bnorm, rn, relres, tol_in;
  int sweep, it, maxit_in, refinements, status;
};

// counters of one step, read back after the launch
struct StepState {
  double s4[4];
  double max_relres;
  int kk, status;
  int picard_iters[3];
  int gmres_iters_total, refinements_total;
};

__device__ __forceinline__ void set_cond(cudaGraphConditionalHandle h, bool v) {
  cudaGraphSetConditional(h, v ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// vector kernels with counts read from device memory
// ---------------------------------------------------------------------------

// partial[b * DSTRIDE + k] = block b's share of v_k . w, where v_k = V_k for
// k < *np + add and the last vector is w itself (same blocking and order as
// k_multidot).  Launch grid (RED_BLOCKS, ceil((restart + 2) / 8)) of 256
// threads (rows past the current count return); returns at once when gate
// != nullptr and *gate == 0.
__global__ void k_ddots(const double* __restrict__ V, const int* __restrict__ np, int add, int64_t n,
                        const double* __restrict__ w, double* __restrict__ partial, const int* __restrict__ gate) {
  if (gate && !*gate) return;
  const int nV = *np + add;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  block_dots_group(
      nV + 1, [&](int k) { return k < nV ? V + (int64_t)k * n : w; }, w, lo, hi,
      [&](int k0) { return partial + (int64_t)blockIdx.x * DSTRIDE + k0; });
}

// out[k] = sum over blocks of partial[b * DSTRIDE + k], k < *np + add + 1
// (block k; launch MAX_RESTART + 2 blocks of 256 threads)
__global__ void k_dreduce(const double* __restrict__ partial, const int* __restrict__ np, int add,
                          double* __restrict__ out, const int* __restrict__ gate) {
  if (gate && !*gate) return;
  const int k = blockIdx.x;
  if (k >= *np + add + 1) return;
  __shared__ double red[256];
  double s = 0.0;
  for (int b = threadIdx.x; b < RED_BLOCKS; b += blockDim.x) s += partial[b * DSTRIDE + k];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[k] = red[0];
}

// w += sum_{k < *np + add} c_k V_k; element pairs when `pairs` (n even, V
// and w 16-byte aligned; launch n/2 threads then), single elements otherwise
__global__ void k_dmultiaxpy(const double* __restrict__ V, const int* __restrict__ np, int add, int64_t n,
                             const double* __restrict__ c, double* __restrict__ w, const int* __restrict__ gate,
                             int pairs) {
  if (gate && !*gate) return;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int nvec = *np + add;
  if (pairs) {
    if (2 * i < n) multiaxpy_pair(V, nvec, n, c, w, i);
    return;
  }
  if (i >= n) return;
  double acc = w[i];
  for (int k = 0; k < nvec; ++k) acc += c[k] * V[(int64_t)k * n + i];
  w[i] = acc;
}

// Z_j = z (j from the state): the flexible GMRES keeps the preconditioned
// vectors for the restart update
__global__ void k_store_col(const double* __restrict__ z, double* __restrict__ Z, const int* __restrict__ j,
                            int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) Z[(int64_t)*j * n + i] = z[i];
}

// V_j = w * inv and the next vmult input xin = V_j (j and inv from the state)
__global__ void k_dnormalize(const double* w, double* V, const GmState* __restrict__ s, int64_t n,
                             double* __restrict__ xin) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = w[i] * s->inv;
  V[(int64_t)s->j * n + i] = v;
  xin[i] = v;
}

// x = 0 where the right-hand side norm is zero
__global__ void k_zero_if(double* __restrict__ x, int64_t n, const double* __restrict__ norm) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && *norm == 0.0) x[i] = 0.0;
}

// ---------------------------------------------------------------------------
// single-thread control kernels (GMRES)
// ---------------------------------------------------------------------------

__global__ void k_gm_begin(GmState* s, double tol, int maxit, int restart, const double* tol_dev,
                           const int* maxit_dev) {
  s->bnorm = sqrt(s->dot[0]);
  s->tol = tol_dev ? *tol_dev : tol;
  s->maxit = maxit_dev ? *maxit_dev : maxit;
  s->restart = restart;
  s->it = 0;
  s->cycles = 0;
  s->jused = 0;
  s->relres = 0.0;
  s->status = isfinite(s->bnorm) ? 0 : DG_ERR_NONFINITE;
}

// after the residual of a cycle: beta, relative residual, continue?
__global__ void k_cycle_end(GmState* s, cudaGraphConditionalHandle h) {
  const double beta = sqrt(s->dot[0]);
  if (!isfinite(beta)) s->status = DG_ERR_NONFINITE;
  s->beta = beta;
  s->relres = s->bnorm > 0.0 ? beta / s->bnorm : 0.0;
  s->cycles++;
  set_cond(h, s->status == 0 && beta > s->tol * s->bnorm && s->it < s->maxit && s->cycles <= s->maxit);
}

__global__ void k_cycle_begin(GmState* s, cudaGraphConditionalHandle h_inner) {
  for (int i = 0; i <= MAX_RESTART; ++i) s->g[i] = 0.0;
  s->g[0] = s->beta;
  s->j = 0;
  s->inv = 1.0 / s->beta;
  set_cond(h_inner, s->status == 0 && s->it < s->maxit);
}

// first classical Gram-Schmidt pass: H(:, j) = V^T w, |w'|^2 = |w|^2 - |h|^2,
// second pass only when the projection cancelled w to |w'| < 1e-3 |w|
__global__ void k_orth1(GmState* s) {
  const int j = s->j, R = s->restart;
  double proj = 0.0;
  for (int k = 0; k <= j; ++k) {
    const double h = s->dot[k];
    s->H[k * R + j] = h;
    s->c[k] = -h;
    proj += h * h;
  }
  s->w2 = s->dot[j + 1] - proj;
  s->reorth = !(s->w2 > 1e-6 * s->dot[j + 1]);
}

__global__ void k_orth2(GmState* s) {
  if (!s->reorth) return;
  const int j = s->j, R = s->restart;
  double proj = 0.0;
  for (int k = 0; k <= j; ++k) {
    const double h = s->dot[k];
    s->H[k * R + j] += h;
    s->c[k] = -h;
    proj += h * h;
  }
  s->w2 = s->dot[j + 1] - proj;
}

// H(j+1, j), Givens rotations, residual estimate; continue the Arnoldi loop?
__global__ void k_arnoldi_end(GmState* s, cudaGraphConditionalHandle h) {
  const int j = s->j, R = s->restart;
  double* H = s->H;
  const double hn = sqrt(s->w2 < 0.0 ? 0.0 : s->w2);
  if (!isfinite(hn)) s->status = DG_ERR_NONFINITE;
  s->inv = hn > 0.0 ? 1.0 / hn : 0.0;
  H[(j + 1) * R + j] = hn;
  for (int k = 0; k < j; ++k) {
    const double t = s->cs[k] * H[k * R + j] + s->sn[k] * H[(k + 1) * R + j];
    H[(k + 1) * R + j] = -s->sn[k] * H[k * R + j] + s->cs[k] * H[(k + 1) * R + j];
    H[k * R + j] = t;
  }
  const double den = hypot(H[j * R + j], H[(j + 1) * R + j]);
  s->cs[j] = H[j * R + j] / den;
  s->sn[j] = H[(j + 1) * R + j] / den;
  H[j * R + j] = den;
  H[(j + 1) * R + j] = 0.0;
  s->g[j + 1] = -s->sn[j] * s->g[j];
  s->g[j] = s->cs[j] * s->g[j];
  s->it++;
  s->jused = j + 1;
  s->j = j + 1;
  const bool conv = fabs(s->g[j + 1]) <= s->tol * s->bnorm;
  set_cond(h, s->status == 0 && !conv && s->it < s->maxit && j + 1 < R);
}

// y = H^-1 g (upper triangular, jused columns)
__global__ void k_solve_y(GmState* s) {
  const int J = s->jused, R = s->restart;
  for (int i = J - 1; i >= 0; --i) {
    double t = s->g[i];
    for (int k = i + 1; k < J; ++k) t -= s->H[i * R + k] * s->y[k];
    s->y[i] = t / s->H[i * R + i];
  }
}

// ---------------------------------------------------------------------------
// control kernels of the refinement sweeps and the Picard loop
// ---------------------------------------------------------------------------

__global__ void k_ir_begin(IrState* r) {
  r->bnorm = sqrt(r->dot0);
  r->sweep = 0;
  r->it = 0;
  r->refinements = 0;
  r->relres = 0.0;
  r->status = isfinite(r->bnorm) ? 0 : DG_ERR_NONFINITE;
}

__global__ void k_ir_check(IrState* r, double rtol, int maxit, double inner_rtol, cudaGraphConditionalHandle h) {
  const double rn = sqrt(r->dot0);
  if (!isfinite(rn)) r->status = DG_ERR_NONFINITE;
  r->rn = rn;
  r->relres = r->bnorm > 0.0 ? rn / r->bnorm : 0.0;
  r->refinements = r->sweep;
  const bool conv = rn <= rtol * r->bnorm;
  const bool cont = r->status == 0 && !conv && r->it < maxit && r->sweep < 60;
  // the inner solve only has to beat the FP32 operator's accuracy
  r->tol_in = fmax(inner_rtol, 0.5 * rtol * r->bnorm / rn);
  r->maxit_in = maxit - r->it;
  r->sweep++;
  set_cond(h, cont);
}

__global__ void k_ir_after(IrState* r, const GmState* s) {
  r->it += s->it;
  if (s->status) r->status = s->status;
}

__global__ void k_step_begin(StepState* ss) {
  for (int k = 0; k < 4; ++k) ss->s4[k] = 0.0;
  ss->max_relres = 0.0;
  ss->kk = 0;
  ss->status = 0;
  for (int l = 0; l < 3; ++l) ss->picard_iters[l] = 0;
  ss->gmres_iters_total = 0;
  ss->refinements_total = 0;
}

__global__ void k_pic_begin(StepState* ss, cudaGraphConditionalHandle h) {
  ss->kk = 0;
  set_cond(h, ss->status == 0);
}

// solve counters of one Picard iteration (gs: plain GMRES, ir: refinement)
__global__ void k_acc_solve(StepState* ss, const GmState* gs, const IrState* ir) {
  if (ir) {
    ss->gmres_iters_total += ir->it;
    ss->refinements_total += ir->refinements;
    if (ir->relres > ss->max_relres) ss->max_relres = ir->relres;
    if (ir->status) ss->status = ir->status;
  } else {
    ss->gmres_iters_total += gs->it;
    if (gs->relres > ss->max_relres) ss->max_relres = gs->relres;
    if (gs->status) ss->status = gs->status;
  }
}

__global__ void k_pic_check(StepState* ss, int l, double rtol, int kmax, int fixed, cudaGraphConditionalHandle h) {
  const double* s4 = ss->s4;
  ss->kk++;
  ss->picard_iters[l] = ss->kk;
  if (!isfinite(s4[0] + s4[1] + s4[2] + s4[3])) ss->status = DG_ERR_NONFINITE;
  const double dp = sqrt(s4[0] / (s4[1] > 0 ? s4[1] : 1e-300));
  const double du = s4[3] > 0 ? sqrt(s4[2] / s4[3]) : 0.0;
  const bool stop = fixed <= 0 && fmax(dp, du) < rtol;
  set_cond(h, ss->status == 0 && ss->kk < kmax && !stop);
}

// ---------------------------------------------------------------------------
// capture helpers
// ---------------------------------------------------------------------------

// a conditional handle of the graph being captured on `st`
static int make_handle(cudaStream_t st, cudaGraphConditionalHandle* h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g;
  DG_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, nullptr, nullptr, nullptr));
  if (cs != cudaStreamCaptureStatusActive) {
    set_error("step graph: stream is not capturing");
    return DG_ERR_CUDA;
  }
  DG_CUDA(cudaGraphConditionalHandleCreate(h, g, 0, cudaGraphCondAssignDefault));
  return DG_OK;
}

// appends a while node on handle h to the capture on `st`; its body is then
// captured on `body` until while_close(body)
static int while_open(cudaStream_t st, cudaStream_t body, cudaGraphConditionalHandle h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  DG_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &ed, &nd));
  cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  DG_CUDA(cudaGraphAddNode(&node, g, deps, ed, nd, &p));
  cudaGraph_t bodyg = p.conditional.phGraph_out[0];
  DG_CUDA(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  DG_CUDA(cudaStreamBeginCaptureToGraph(body, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  return DG_OK;
}

static int while_close(cudaStream_t body) {
  cudaGraph_t g;
  DG_CUDA(cudaStreamEndCapture(body, &g));
  return DG_OK;
}

}  // namespace dg

// cached executable graph of one step configuration
struct StepGraph {
  static constexpr int kStreams = 5;
  cudaStream_t s[kStreams] = {};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  dg::StepState* host = nullptr;   // pinned read-back of the counters
  unsigned char key[2048];
  size_t key_len = 0;
  bool valid = false;
};

namespace dg {

void graph_release(dg_mesh* m) {
  StepGraph* G = m->graph;
  if (!G) return;
  if (G->exec) cudaGraphExecDestroy(G->exec);
  if (G->graph) cudaGraphDestroy(G->graph);
  for (auto& s : G->s)
    if (s) cudaStreamDestroy(s);
  if (G->host) cudaFreeHost(G->host);
  delete G;
  m->graph = nullptr;
}

namespace {

struct Work {
  StepState* ss;
  IrState* ir;
  GmState* gs64;   // plain FP64 solve
  GmState* gs32;   // inner solve of the refinement sweeps
  double* xin;
  double* w;
  double* tmp;
  double* partial;   // RED_BLOCKS x DSTRIDE
};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

int ensure_work(dg_mesh* m, Work* wk) {
  const size_t o1 = align256(sizeof(StepState)), o2 = o1 + align256(sizeof(IrState)),
               o3 = o2 + align256(sizeof(GmState)), o4 = o3 + align256(sizeof(GmState));
  int rc;
  if ((rc = m->gstate.ensure(o4)) != DG_OK) return rc;
  const int64_t n = m->N;
  if ((rc = m->gwork.ensure(sizeof(double) * (3 * n + (int64_t)RED_BLOCKS * DSTRIDE))) != DG_OK) return rc;
  char* b = m->gstate.as<char>();
  wk->ss = reinterpret_cast<StepState*>(b);
  wk->ir = reinterpret_cast<IrState*>(b + o1);
  wk->gs64 = reinterpret_cast<GmState*>(b + o2);
  wk->gs32 = reinterpret_cast<GmState*>(b + o3);
  double* v = m->gwork.as<double>();
  wk->xin = v;
  wk->w = v + n;
  wk->tmp = v + 2 * n;
  wk->partial = v + 3 * n;
  return DG_OK;
}

// out = v . v reduced in the fixed order of the host-driven solver
int dot_self(dg_mesh* m, const Work& wk, const double* v, double* out, cudaStream_t st) {
  k_multidot<<<RED_BLOCKS, 256, 0, st>>>(v, 1, m->N, v, wk.partial);
  k_reduce_partials<<<1, 256, 0, st>>>(wk.partial, 1, RED_BLOCKS, out);
  DG_LAUNCH_CHECK("graph dot");
  return DG_OK;
}

// Restarted GMRES(restart) on A, as the host-driven solver computes it, with
// the loops as while nodes.  Capture streams: s[0] current, s[1] restart
// cycles, s[2] Arnoldi steps.
int capture_gmres(dg_mesh* m, const Work& wk, GmState* gs, const Vmult& A, const double* b, double* x,
                  bool x_is_zero, double tol, int maxit, int restart, const double* tol_dev, const int* maxit_dev,
                  const cudaStream_t* s, bool pc = false) {
  const int64_t n = m->N;
  int rc;
  if ((rc = m->gm_V.ensure(sizeof(double) * (size_t)(restart + 1) * n)) != DG_OK) return rc;
  double* V = m->gm_V.as<double>();
  // flexible right preconditioning as in the host-driven solver: Z_j =
  // P^-1 V_j (restart columns), the preconditioned vector of the current
  // step in the column after them
  if (pc && (rc = m->gm_pc.ensure(sizeof(double) * (size_t)(restart + 1) * n)) != DG_OK) return rc;
  double* Z = pc ? m->gm_pc.as<double>() : nullptr;
  double* zt = pc ? Z + (int64_t)restart * n : nullptr;
  const unsigned gb = grid_for(n, 256);
  // k_dmultiaxpy over element pairs when every target allows 16-byte access
  const int pairs = n % 2 == 0 && ((uintptr_t)V & 15) == 0 && ((uintptr_t)wk.w & 15) == 0 &&
                    ((uintptr_t)x & 15) == 0 && (!pc || ((uintptr_t)Z & 15) == 0);
  const unsigned gma = grid_for(pairs ? n / 2 : n, 256);
  const dim3 dgrid(RED_BLOCKS, (restart + 2 + 7) / 8);   // k_ddots: up to restart + 1 vectors and w
  if ((rc = dot_self(m, wk, b, &gs->dot[0], s[0])) != DG_OK) return rc;
  k_gm_begin<<<1, 1, 0, s[0]>>>(gs, tol, maxit, restart, tol_dev, maxit_dev);
  k_zero_if<<<gb, 256, 0, s[0]>>>(x, n, &gs->bnorm);
  if (x_is_zero) {
    DG_CUDA(cudaMemcpyAsync(V, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s[0]));
  } else {
    if ((rc = A(x, wk.tmp, s[0])) != DG_OK) return rc;
    k_axpby<<<gb, 256, 0, s[0]>>>(n, 1.0, b, -1.0, wk.tmp, V);
  }
  if ((rc = dot_self(m, wk, V, &gs->dot[0], s[0])) != DG_OK) return rc;
  cudaGraphConditionalHandle hc, ha;
  if ((rc = make_handle(s[0], &hc)) != DG_OK) return rc;
  k_cycle_end<<<1, 1, 0, s[0]>>>(gs, hc);
  if ((rc = while_open(s[0], s[1], hc)) != DG_OK) return rc;
  {
    if ((rc = make_handle(s[1], &ha)) != DG_OK) return rc;
    k_cycle_begin<<<1, 1, 0, s[1]>>>(gs, ha);
    k_dnormalize<<<gb, 256, 0, s[1]>>>(V, V, gs, n, wk.xin);
    if ((rc = while_open(s[1], s[2], ha)) != DG_OK) return rc;
    {
      cudaStream_t sa = s[2];
      if (pc) {
        if ((rc = precond_apply(m, wk.xin, zt, sa)) != DG_OK) return rc;
        k_store_col<<<gb, 256, 0, sa>>>(zt, Z, &gs->j, n);
        if ((rc = A(zt, wk.w, sa)) != DG_OK) return rc;
      } else if ((rc = A(wk.xin, wk.w, sa)) != DG_OK) {
        return rc;
      }
      k_ddots<<<dgrid, 256, 0, sa>>>(V, &gs->j, 1, n, wk.w, wk.partial, nullptr);
      k_dreduce<<<MAX_RESTART + 2, 256, 0, sa>>>(wk.partial, &gs->j, 1, gs->dot, nullptr);
      k_orth1<<<1, 1, 0, sa>>>(gs);
      k_dmultiaxpy<<<gma, 256, 0, sa>>>(V, &gs->j, 1, n, gs->c, wk.w, nullptr, pairs);
      k_ddots<<<dgrid, 256, 0, sa>>>(V, &gs->j, 1, n, wk.w, wk.partial, &gs->reorth);
      k_dreduce<<<MAX_RESTART + 2, 256, 0, sa>>>(wk.partial, &gs->j, 1, gs->dot, &gs->reorth);
      k_orth2<<<1, 1, 0, sa>>>(gs);
      k_dmultiaxpy<<<gma, 256, 0, sa>>>(V, &gs->j, 1, n, gs->c, wk.w, &gs->reorth, pairs);
      k_arnoldi_end<<<1, 1, 0, sa>>>(gs, ha);
      k_dnormalize<<<gb, 256, 0, sa>>>(wk.w, V, gs, n, wk.xin);
      DG_LAUNCH_CHECK("graph arnoldi step");
    }
    if ((rc = while_close(s[2])) != DG_OK) return rc;
    k_solve_y<<<1, 1, 0, s[1]>>>(gs);
    k_dmultiaxpy<<<gma, 256, 0, s[1]>>>(pc ? Z : V, &gs->jused, 0, n, gs->y, x, nullptr, pairs);
    if ((rc = A(x, wk.tmp, s[1])) != DG_OK) return rc;
    k_axpby<<<gb, 256, 0, s[1]>>>(n, 1.0, b, -1.0, wk.tmp, V);
    if ((rc = dot_self(m, wk, V, &gs->dot[0], s[1])) != DG_OK) return rc;
    k_cycle_end<<<1, 1, 0, s[1]>>>(gs, hc);
    DG_LAUNCH_CHECK("graph restart cycle");
  }
  return while_close(s[1]);
}

// Iterative refinement (FP64 residual, inner GMRES on the FP32 operator).
// Capture streams: s[0] current, s[1] sweeps, s[2..3] inner GMRES.
int capture_gmres_ir(dg_mesh* m, const Work& wk, const Vmult& A64, const Vmult& A32, const double* b, double* x,
                     double rtol, int restart, int maxit, double inner_rtol, const cudaStream_t* s,
                     bool pc = false) {
  const int64_t n = m->N;
  int rc;
  if ((rc = m->irw.ensure(sizeof(double) * 2 * n)) != DG_OK) return rc;
  double* r = m->irw.as<double>();
  double* d = r + n;
  IrState* ir = wk.ir;
  const unsigned gb = grid_for(n, 256);
  if (!(inner_rtol > 0.0)) inner_rtol = 1e-4;
  if ((rc = dot_self(m, wk, b, &ir->dot0, s[0])) != DG_OK) return rc;
  k_ir_begin<<<1, 1, 0, s[0]>>>(ir);
  k_zero_if<<<gb, 256, 0, s[0]>>>(x, n, &ir->bnorm);
  if ((rc = A64(x, r, s[0])) != DG_OK) return rc;
  k_axpby<<<gb, 256, 0, s[0]>>>(n, 1.0, b, -1.0, r, r);
  if ((rc = dot_self(m, wk, r, &ir->dot0, s[0])) != DG_OK) return rc;
  cudaGraphConditionalHandle h;
  if ((rc = make_handle(s[0], &h)) != DG_OK) return rc;
  k_ir_check<<<1, 1, 0, s[0]>>>(ir, rtol, maxit, inner_rtol, h);
  if ((rc = while_open(s[0], s[1], h)) != DG_OK) return rc;
  {
    DG_CUDA(cudaMemsetAsync(d, 0, sizeof(double) * n, s[1]));
    if ((rc = capture_gmres(m, wk, wk.gs32, A32, r, d, true, 0.0, 0, restart, &ir->tol_in, &ir->maxit_in,
                            s + 1, pc)) != DG_OK)
      return rc;
    k_ir_after<<<1, 1, 0, s[1]>>>(ir, wk.gs32);
    k_axpby<<<gb, 256, 0, s[1]>>>(n, 1.0, x, 1.0, d, x);
    if ((rc = A64(x, r, s[1])) != DG_OK) return rc;
    k_axpby<<<gb, 256, 0, s[1]>>>(n, 1.0, b, -1.0, r, r);
    if ((rc = dot_self(m, wk, r, &ir->dot0, s[1])) != DG_OK) return rc;
    k_ir_check<<<1, 1, 0, s[1]>>>(ir, rtol, maxit, inner_rtol, h);
    DG_LAUNCH_CHECK("graph refinement sweep");
  }
  return while_close(s[1]);
}

// the whole ARK2 step, as step_host computes it, on capture stream s[0]
int capture_step(dg_mesh* m, const dg_phys* ph, double* q, double dt, const dg_step_opts* o, const Work& wk,
                 const cudaStream_t* s) {
  const int64_t n = m->N;
  const Ark2 tab;
  int rc;
  if ((rc = m->fns.ensure(sizeof(double) * 15 * n)) != DG_OK) return rc;
  if ((rc = m->fs.ensure(sizeof(double) * 12 * n)) != DG_OK) return rc;
  if ((rc = m->st.ensure(sizeof(double) * 19 * n)) != DG_OK) return rc;
  Red red;
  if ((rc = ensure_red(m, &red)) != DG_OK) return rc;
  double* Fns[3] = {m->fns.as<double>(), m->fns.as<double>() + 5 * n, m->fns.as<double>() + 10 * n};
  double* Fs[3] = {m->fs.as<double>(), m->fs.as<double>() + 4 * n, m->fs.as<double>() + 8 * n};
  double* ws = m->st.as<double>();
  double* y = ws;
  double* rho = ws + 5 * n;
  double* mhat = ws + 6 * n;
  double* ehat = ws + 9 * n;
  double* u = ws + 10 * n;
  double* unew = ws + 13 * n;
  double* p = ws + 16 * n;
  double* pnew = ws + 17 * n;
  double* rhs = ws + 18 * n;
  const unsigned gb = grid_for(n, 256);
  const bool pairs = ph->precision == DG_PAIRS;
  const bool mixed = ph->precision != DG_FP64 && !pairs;
  const bool incr = ph->precision == DG_MIXED_EXPLICIT && !m->bg_set;
  const PhysK pk{ph->gamma, ph->g, ph->f, ph->f_cell, ph->lambda_min};
  const bool pc = o->gmres.precond != DG_PRECOND_NONE;
  k_step_begin<<<1, 1, 0, s[0]>>>(wk.ss);
  if ((rc = explicit_rt(m, ph, q, Fns[0], Fs[0], s[0])) != DG_OK) return rc;
  if (incr && (rc = increment_begin(m, ph->gamma, q, s[0])) != DG_OK) return rc;
  const double* yprev = q;
  for (int l = 1; l <= 2; ++l) {
    const double adt = tab.at[l][l] * dt;
    StageCoefs sc{};
    sc.nst = l;
    sc.dt = dt;
    for (int j = 0; j < l; ++j) {
      sc.fns[j] = Fns[j];
      sc.fs[j] = Fs[j];
      sc.a[j] = tab.a[l][j];
      sc.at[j] = tab.at[l][j];
    }
    k_stage_predict<<<gb, 256, 0, s[0]>>>(q, n, sc, rho, mhat, ehat);
    k_primitives<<<gb, 256, 0, s[0]>>>(yprev, n, ph->gamma, u, p);
    DG_LAUNCH_CHECK("graph stage predictors");
    ImplK k = impl_consts(ph, adt);
    const int kmax = o->picard_fixed > 0 ? o->picard_fixed : o->picard_maxit;
    // preconditioner factored once per stage from the first Picard iterate's
    // coefficients, as the host-driven step does
    if (pc) {
      if ((rc = prepare_rt(m, k, rho, p, u, ph->penalty, s[0])) != DG_OK) return rc;
      if ((rc = precond_setup(m, o->gmres.precond, k, p, ph->penalty, s[0])) != DG_OK) return rc;
    }
    cudaGraphConditionalHandle h;
    if ((rc = make_handle(s[0], &h)) != DG_OK) return rc;
    k_pic_begin<<<1, 1, 0, s[0]>>>(wk.ss, h);
    if ((rc = while_open(s[0], s[1], h)) != DG_OK) return rc;
    {
      cudaStream_t sp = s[1];
      if ((rc = prepare_rt(m, k, rho, p, u, ph->penalty, sp)) != DG_OK) return rc;
      if ((rc = rhs_rt(m, k, rho, p, u, mhat, ehat, rhs, sp)) != DG_OK) return rc;
      DG_CUDA(cudaMemcpyAsync(pnew, p, sizeof(double) * n, cudaMemcpyDeviceToDevice, sp));
      SchurCtx schur{m, k, rho, p, ph->penalty};
      Vmult A = make_vmult(&schur);
      if (mixed) {
        Schur32Ctx sc32;
        if ((rc = prepare32(m, k, rho, p, u, ph->penalty, sp, &sc32)) != DG_OK) return rc;
        Vmult A32 = make_vmult32(&sc32);
        if ((rc = capture_gmres_ir(m, wk, A, A32, rhs, pnew, o->gmres.rtol, o->gmres.restart, o->gmres.maxit,
                                   o->gmres.inner_rtol, s + 1, pc)) != DG_OK)
          return rc;
        k_acc_solve<<<1, 1, 0, sp>>>(wk.ss, nullptr, wk.ir);
      } else {
        // DG_PAIRS: the same FP64 GMRES around the pair vmult
        SchurDfCtx sdf;
        if (pairs) {
          if ((rc = prepare_pairs(m, k, rho, p, u, ph->penalty, sp, &sdf)) != DG_OK) return rc;
          A = make_vmult_pairs(&sdf);
        }
        if ((rc = capture_gmres(m, wk, wk.gs64, A, rhs, pnew, false, o->gmres.rtol, o->gmres.maxit,
                                o->gmres.restart, nullptr, nullptr, s + 1, pc)) != DG_OK)
          return rc;
        k_acc_solve<<<1, 1, 0, sp>>>(wk.ss, wk.gs64, nullptr);
      }
      if ((rc = recover_rt(m, k, rho, u, mhat, pnew, unew, sp)) != DG_OK) return rc;
      k_picard_norms<<<RED_BLOCKS, 256, 0, sp>>>(p, pnew, u, unew, n, red.partial);
      k_reduce_partials<<<4, 256, 0, sp>>>(red.partial, 4, RED_BLOCKS, wk.ss->s4);
      k_pic_check<<<1, 1, 0, sp>>>(wk.ss, l, o->picard_rtol, kmax, o->picard_fixed, h);
      DG_CUDA(cudaMemcpyAsync(p, pnew, sizeof(double) * n, cudaMemcpyDeviceToDevice, sp));
      DG_CUDA(cudaMemcpyAsync(u, unew, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, sp));
      DG_LAUNCH_CHECK("graph picard iteration");
    }
    if ((rc = while_close(s[1])) != DG_OK) return rc;
    k_stage_state<<<gb, 256, 0, s[0]>>>(rho, u, p, n, ph->gamma, y);
    DG_LAUNCH_CHECK("graph stage state");
    if (incr) {
      rc = explicit_increment(m, pk, y, q, Fns[0], Fs[0], Fns[l], Fs[l], s[0]);
      // Fns[0] already holds the damping at q: add its increment only
      if (rc == DG_OK) rc = sponge_rt(m, y, Fns[l], s[0], q);
    } else {
      rc = explicit_rt(m, ph, y, Fns[l], Fs[l], s[0]);
    }
    if (rc != DG_OK) return rc;
    yprev = y;
  }
  StageCoefs fin{};
  fin.nst = 3;
  fin.dt = dt;
  for (int j = 0; j < 3; ++j) {
    fin.fns[j] = Fns[j];
    fin.fs[j] = Fs[j];
    fin.a[j] = tab.b[j];
  }
  k_final_update<<<gb, 256, 0, s[0]>>>(q, n, fin, &wk.ss->status);
  DG_LAUNCH_CHECK("graph final update");
  return DG_OK;
}

// everything the captured kernels depend on
size_t make_key(const dg_mesh* m, const dg_phys* ph, const double* q, double dt, const dg_step_opts* o,
                unsigned char* out) {
  struct Key {
    const double* q;
    double dt, gamma, g, f, lambda_min;
    const double* fcell;
    int variant, penalty, precision, bg_set, sponge_set;
    double picard_rtol;
    int picard_maxit, picard_fixed;
    double rtol, inner_rtol;
    int restart, maxit, precond;
    int tile[K_COUNT], tile32[K_COUNT], tilep[K_COUNT], fused_stage[3];
    const void* bp[dg_mesh::kBufs];
    size_t bb[dg_mesh::kBufs];
  } k;
  static_assert(sizeof(Key) <= sizeof(StepGraph::key), "graph key too large");
  std::memset(&k, 0, sizeof(k));
  k.q = q;
  k.dt = dt;
  k.gamma = ph->gamma;
  k.g = ph->g;
  k.f = ph->f;
  k.lambda_min = ph->lambda_min;
  k.fcell = ph->f_cell;
  k.variant = ph->variant;
  k.penalty = ph->penalty;
  k.precision = ph->precision;
  k.bg_set = m->bg_set ? 1 : 0;
  k.sponge_set = m->sponge_set ? 1 : 0;
  k.picard_rtol = o->picard_rtol;
  k.picard_maxit = o->picard_maxit;
  k.picard_fixed = o->picard_fixed;
  k.rtol = o->gmres.rtol;
  k.inner_rtol = o->gmres.inner_rtol;
  k.restart = o->gmres.restart;
  k.maxit = o->gmres.maxit;
  k.precond = o->gmres.precond;
  for (int i = 0; i < K_COUNT; ++i) {
    k.tile[i] = m->tile[i];
    k.tile32[i] = m->tile32[i];
    k.tilep[i] = m->tilep[i];
  }
  for (int i = 0; i < 3; ++i) k.fused_stage[i] = m->fused_stage[i];
  const DBuf* b[dg_mesh::kBufs];
  m->bufs(b);
  for (int i = 0; i < dg_mesh::kBufs; ++i) {
    k.bp[i] = b[i]->p;
    k.bb[i] = b[i]->bytes;
  }
  std::memcpy(out, &k, sizeof(k));
  return sizeof(k);
}

void drop_graph(StepGraph* G) {
  if (G->exec) cudaGraphExecDestroy(G->exec);
  if (G->graph) cudaGraphDestroy(G->graph);
  G->exec = nullptr;
  G->graph = nullptr;
  G->valid = false;
}

// capture the step into G (buffers already sized); false when the buffers
// moved during the capture
int capture(dg_mesh* m, const dg_phys* ph, double* q, double dt, const dg_step_opts* o, StepGraph* G,
            bool* stable) {
  Work wk;
  int rc;
  if ((rc = ensure_work(m, &wk)) != DG_OK) return rc;
  unsigned char before[sizeof(StepGraph::key)];
  const size_t kl = make_key(m, ph, q, dt, o, before);
  drop_graph(G);
  DG_CUDA(cudaStreamBeginCapture(G->s[0], cudaStreamCaptureModeRelaxed));
  int crc = capture_step(m, ph, q, dt, o, wk, G->s);
  if (crc != DG_OK) {
    // close body captures left open by the error, innermost first
    for (int i = StepGraph::kStreams - 1; i >= 1; --i) {
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(G->s[i], &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        cudaGraph_t gb = nullptr;
        cudaStreamEndCapture(G->s[i], &gb);
      }
    }
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(G->s[0], &g);
  if (crc != DG_OK) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return crc;
  }
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(e, "step graph capture");
  }
  G->graph = g;
  unsigned char after[sizeof(StepGraph::key)];
  make_key(m, ph, q, dt, o, after);
  *stable = std::memcmp(before, after, kl) == 0;
  if (!*stable) {
    drop_graph(G);
    return DG_OK;
  }
  DG_CUDA(cudaGraphInstantiate(&G->exec, G->graph, 0));
  std::memcpy(G->key, after, kl);
  G->key_len = kl;
  G->valid = true;
  return DG_OK;
}

int graph_of(dg_mesh* m, StepGraph** out) {
  if (!m->graph) {
    StepGraph* G = new StepGraph();
    m->graph = G;
    for (auto& s : G->s) DG_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    DG_CUDA(cudaMallocHost(&G->host, sizeof(StepState)));
  }
  *out = m->graph;
  return DG_OK;
}

// One host-driven step on a copy of q sizes every workspace and builds the
// one-time data (FP32 geometry, background rates), so that a capture
// allocates nothing; captures check that.
int warm_up(dg_mesh* m, const dg_phys* ph, const double* q, double dt, const dg_step_opts* o, cudaStream_t st) {
  double* qs = nullptr;
  DG_CUDA(cudaMalloc(&qs, sizeof(double) * 5 * m->N));
  cudaError_t e = cudaMemcpyAsync(qs, q, sizeof(double) * 5 * m->N, cudaMemcpyDeviceToDevice, st);
  int rc = e == cudaSuccess ? step_host(m, ph, qs, dt, o, nullptr, st) : DG_OK;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(qs);
  if (e != cudaSuccess) return cuda_fail(e, "step graph warm-up");
  if (rc != DG_OK && rc != DG_ERR_NOT_CONVERGED) return rc;
  return DG_OK;
}

int fill_info(const StepState& h, dg_step_info* info) {
  if (info) {
    dg_step_info inf{};
    for (int l = 0; l < 3; ++l) inf.picard_iters[l] = h.picard_iters[l];
    inf.gmres_iters_total = h.gmres_iters_total;
    inf.max_relres = h.max_relres;
    inf.refinements_total = h.refinements_total;
    *info = inf;
  }
  if (h.status == DG_ERR_NONFINITE) {
    set_error("imex_ark2_step: non-finite value in the Krylov or Picard iteration (state left unchanged)");
    return DG_ERR_NONFINITE;
  }
  return h.status;
}

}  // namespace

int step_graph(dg_mesh* m, const dg_phys* ph, double* q, double dt, const dg_step_opts* o, dg_step_info* info,
               cudaStream_t st) {
  if (m->prof.on) {
    set_error("imex_ark2_step: graph mode does not run under dg_profile_begin");
    return DG_ERR_UNSUPPORTED;
  }
  int rc;
  StepGraph* G;
  if ((rc = graph_of(m, &G)) != DG_OK) return rc;
  unsigned char key[sizeof(StepGraph::key)];
  const size_t kl = make_key(m, ph, q, dt, o, key);
  if (!G->valid || G->key_len != kl || std::memcmp(G->key, key, kl) != 0) {
    if ((rc = warm_up(m, ph, q, dt, o, st)) != DG_OK) return rc;
    bool stable = false;
    if ((rc = capture(m, ph, q, dt, o, G, &stable)) != DG_OK) return rc;
    if (!stable) {
      set_error("imex_ark2_step: workspace moved during graph capture");
      return DG_ERR_CUDA;
    }
  }
  DG_CUDA(cudaGraphLaunch(G->exec, st));
  Work wk;
  if ((rc = ensure_work(m, &wk)) != DG_OK) return rc;
  DG_CUDA(cudaMemcpyAsync(G->host, wk.ss, sizeof(StepState), cudaMemcpyDeviceToHost, st));
  DG_CUDA(cudaStreamSynchronize(st));
  return fill_info(*G->host, info);
}

}  // namespace dg

// ---------------------------------------------------------------------------
// several meshes in one graph (ensemble groups): the steps are captured as
// parallel branches of one graph, so an ensemble step is one launch
// ---------------------------------------------------------------------------

struct MultiGraph {
  cudaStream_t main = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<unsigned char> key;
  bool valid = false;
};

namespace dg {

void multi_graph_release(MultiGraph* M) {
  if (!M) return;
  if (M->exec) cudaGraphExecDestroy(M->exec);
  if (M->graph) cudaGraphDestroy(M->graph);
  if (M->main) cudaStreamDestroy(M->main);
  if (M->fork) cudaEventDestroy(M->fork);
  for (auto ev : M->join) cudaEventDestroy(ev);
  delete M;
}

int multi_step_graph(int ng, dg_mesh* const* meshes, const dg_phys* phs, double* const* qs, const double* dts,
                     const dg_step_opts* o, dg_step_info* infos, MultiGraph** cache, cudaStream_t st) {
  int rc;
  if (!*cache) {
    MultiGraph* M = new MultiGraph();
    *cache = M;
    DG_CUDA(cudaStreamCreateWithFlags(&M->main, cudaStreamNonBlocking));
    DG_CUDA(cudaEventCreateWithFlags(&M->fork, cudaEventDisableTiming));
  }
  MultiGraph* M = *cache;
  while ((int)M->join.size() < ng) {
    cudaEvent_t ev;
    DG_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    M->join.push_back(ev);
  }
  std::vector<StepGraph*> G(ng);
  std::vector<unsigned char> key;
  for (int k = 0; k < ng; ++k) {
    if (meshes[k]->prof.on) {
      set_error("dg_ensemble_step: graph mode does not run under dg_profile_begin");
      return DG_ERR_UNSUPPORTED;
    }
    if ((rc = graph_of(meshes[k], &G[k])) != DG_OK) return rc;
    unsigned char kk[sizeof(StepGraph::key)];
    const size_t kl = make_key(meshes[k], &phs[k], qs[k], dts[k], o, kk);
    key.insert(key.end(), kk, kk + kl);
  }
  if (!M->valid || M->key != key) {
    for (int k = 0; k < ng; ++k)
      if ((rc = warm_up(meshes[k], &phs[k], qs[k], dts[k], o, st)) != DG_OK) return rc;
    if (M->exec) cudaGraphExecDestroy(M->exec);
    if (M->graph) cudaGraphDestroy(M->graph);
    M->exec = nullptr;
    M->graph = nullptr;
    M->valid = false;
    std::vector<Work> wk(ng);
    for (int k = 0; k < ng; ++k)
      if ((rc = ensure_work(meshes[k], &wk[k])) != DG_OK) return rc;
    std::vector<unsigned char> before;
    for (int k = 0; k < ng; ++k) {
      unsigned char kk[sizeof(StepGraph::key)];
      const size_t kl = make_key(meshes[k], &phs[k], qs[k], dts[k], o, kk);
      before.insert(before.end(), kk, kk + kl);
    }
    DG_CUDA(cudaStreamBeginCapture(M->main, cudaStreamCaptureModeRelaxed));
    int crc = cudaEventRecord(M->fork, M->main) == cudaSuccess ? DG_OK : DG_ERR_CUDA;
    for (int k = 0; k < ng && crc == DG_OK; ++k) {
      StepGraph* g = G[k];
      if (cudaStreamWaitEvent(g->s[0], M->fork, 0) != cudaSuccess) {
        crc = DG_ERR_CUDA;
        break;
      }
      crc = capture_step(meshes[k], &phs[k], qs[k], dts[k], o, wk[k], g->s);
      if (crc == DG_OK && (cudaEventRecord(M->join[k], g->s[0]) != cudaSuccess ||
                           cudaStreamWaitEvent(M->main, M->join[k], 0) != cudaSuccess))
        crc = DG_ERR_CUDA;
    }
    if (crc != DG_OK) {
      // close every capture still open (bodies first), then the main one
      for (int k = 0; k < ng; ++k)
        for (int i = StepGraph::kStreams - 1; i >= 0; --i) {
          cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
          if (cudaStreamIsCapturing(G[k]->s[i], &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive &&
              i > 0) {
            cudaGraph_t gb = nullptr;
            cudaStreamEndCapture(G[k]->s[i], &gb);
          }
        }
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(M->main, &g);
    if (crc != DG_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      if (crc != DG_OK) return crc;
      return cuda_fail(e, "ensemble graph capture");
    }
    M->graph = g;
    std::vector<unsigned char> after;
    for (int k = 0; k < ng; ++k) {
      unsigned char kk[sizeof(StepGraph::key)];
      const size_t kl = make_key(meshes[k], &phs[k], qs[k], dts[k], o, kk);
      after.insert(after.end(), kk, kk + kl);
    }
    if (after != before) {
      set_error("dg_ensemble_step: workspace moved during graph capture");
      return DG_ERR_CUDA;
    }
    DG_CUDA(cudaGraphInstantiate(&M->exec, M->graph, 0));
    M->key = after;
    M->valid = true;
  }
  DG_CUDA(cudaGraphLaunch(M->exec, st));
  for (int k = 0; k < ng; ++k) {
    Work wk;
    if ((rc = ensure_work(meshes[k], &wk)) != DG_OK) return rc;
    DG_CUDA(cudaMemcpyAsync(G[k]->host, wk.ss, sizeof(StepState), cudaMemcpyDeviceToHost, st));
  }
  DG_CUDA(cudaStreamSynchronize(st));
  int out = DG_OK;
  for (int k = 0; k < ng; ++k) {
    const int r = fill_info(*G[k]->host, infos ? &infos[k] : nullptr);
    if (r != DG_OK && out == DG_OK) out = r;
  }
  return out;
}

}  // namespace dg
