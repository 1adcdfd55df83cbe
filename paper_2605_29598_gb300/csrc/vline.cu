// Vertical-line preconditioner of the scaled Schur system (not in the
// paper, whose GMRES runs unpreconditioned; an optional right
// preconditioner for tall, thin cells where the vertical acoustic and
// gravity terms of the Helmholtz operator dominate its conditioning).
//
// The operator of Section 3.1 is y = x + P x - c_g G_z x - c_d Div(h rho w),
// w = rho^{-1} G x.  Along every line of nodes that runs vertically through
// a chain of cells (cells linked by conforming faces xi_d = 1 / xi_d = 0 of
// the last reference direction) the preconditioner keeps only the terms
// that couple nodes of that line: the K_dd metric entry of the vertical
// gradient and divergence, the z component of the face normals, and the
// penalty P of the vertical faces.  With w_z kept as an unknown this is a
// block-tridiagonal system in the unknowns (x, w_z) of one cell line (2n x
// 2n blocks, n = r + 1 nodes per cell line):
//   x + P x - c_g G_z x - c_d D_z(h w_z) = b,   w_z - rho^{-1} G_z x = 0,
// factored by block Thomas in FP32 (Gauss-Jordan inverses with partial
// pivoting) by a group of 2n (rounded up to a power of two) threads per
// line, one block row per thread.  The unknown w_z is carried as alpha w_z,
// alpha = sqrt(c_d h rho rho) at the line's first node, which balances the
// x-w and w-x couplings (their entries differ by ~1e7 otherwise, and the
// unscaled 2n x 2n blocks lose most FP32 digits).  Only chains that end in
// walls at both ends are factored; the lines of other chains (cut by a 2:1
// face, or a vertically periodic column) are left unpreconditioned
// (identity).
#include "solver.cuh"

namespace dg {

namespace {

// z component of n dS, penalty coefficient and face kind of every slot:
// kind 0 wall, 1 conforming interior face, 2 fine side of a 2:1 face (and,
// left from the prefill, the coarse side of one)
__global__ void k_vl_slots(FaceTopo ft, int dim, const double* __restrict__ pcoef, float* __restrict__ nz,
                           float* __restrict__ pc, int8_t* __restrict__ kind) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= ft.nF) return;
  const int sm = ft.fp_minus[p], code = ft.fp_plus[p];
  const float n = (float)ft.fgeo[(int64_t)(dim - 1) * ft.nF + p];
  const float c = pcoef ? (float)pcoef[p] : 0.f;
  nz[sm] = n;
  pc[sm] = c;
  kind[sm] = code == -1 ? 0 : (code >= 0 ? 1 : 2);
  if (code >= 0) {
    nz[code] = -n;
    pc[code] = c;
    kind[code] = 1;
  }
}

// row of a block: M floats from an 8-byte aligned address
template <int M>
__device__ __forceinline__ void load_row(const float* __restrict__ in, float (&row)[M]) {
#pragma unroll
  for (int q = 0; q < M; q += 2) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(in) + q / 2);
    row[q] = v.x;
    row[q + 1] = v.y;
  }
}

struct VlArgs {
  const int* above;
  const int* below;
  const int* heads;
  int64_t nchain, E;
  const float* nz;
  const float* pc;
  const int8_t* kind;
  uint8_t* vfull;          // 1: the chain is factored
  float* fac;              // per line cell (e nfp + t): 3 row-major (2n)^2 blocks Dinv, L Dinv_prev, U
  float* scr;              // per line cell: 2n floats of the forward sweep
  const double* K;         // d*d x N metric (K_dd used)
  const double* invM;      // N
  const double* irho;      // N
  const double* trh;       // S : traces of h rho = gamma p_lag / (gamma - 1)
  const double* plag;      // N
  float hscale, cd, cg;    // gamma/(gamma-1), (gamma-1) a_dt^2, (gamma-1) a_dt^2 g (R2) or 0
};

// value of a 1D table entry at a runtime index, by unrolled selects (a
// dynamic index into the kernel parameters would copy them to local memory)
template <int N>
__device__ __forceinline__ float pick(const float (&v)[MAX_N], int k) {
  float r = v[0];
#pragma unroll
  for (int i = 1; i < N; ++i)
    if (i == k) r = v[i];
  return r;
}

// A group of G >= 2n threads per (chain, horizontal node position t); thread
// p owns row p of the cell blocks (rows >= 2n idle).  For every cell of the
// line it assembles its rows of the diagonal, lower and upper blocks and runs
// the forward sweep of block Thomas -- the products L D'^{-1}_prev and
// (L D'^{-1}_prev) U_prev and the Gauss-Jordan inverse with partial pivoting
// exchange rows by shuffles in the group -- and stores its rows of D'^{-1},
// L D'^{-1}_prev and U.
template <int DIM, int N>
__global__ void __launch_bounds__(256) k_vl_setup(VlArgs a, Tables<float> tb) {
  constexpr int NFP = ipow(N, DIM - 1), NP = ipow(N, DIM), NF = 2 * DIM, M2 = 2 * N, BS = M2 * M2;
  constexpr int G = M2 <= 4 ? 4 : (M2 <= 8 ? 8 : 16);
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t line = gid / G;
  const int p = (int)(gid % G);
  if (line >= a.nchain * NFP) return;      // whole groups: G divides the block
  const int64_t c = line / NFP;
  const int t = (int)(line % NFP);
  const unsigned lane = threadIdx.x & 31u;
  const unsigned gmask = (G == 32 ? 0xffffffffu : ((1u << G) - 1u)) << (lane & ~(unsigned)(G - 1));
  const bool row = p < M2;
  const int pr = row ? p : 0;
  const bool xrow = pr < N;                 // x equation of node k, else w equation of node k
  const int k = xrow ? pr : pr - N;
  const int fb = 2 * (DIM - 1), ftp = fb + 1;
  const int64_t Nn = a.E * NP;
  const int head = a.heads[c];
  int tail = head;
  int64_t len = 1;
  while (a.above[tail] >= 0 && len < a.E) {
    tail = a.above[tail];
    ++len;
  }
  const bool full = a.kind[((int64_t)head * NF + fb) * NFP + t] == 0 &&
                    a.kind[((int64_t)tail * NF + ftp) * NFP + t] == 0;
  if (t == 0 && p == 0) a.vfull[c] = full ? 1 : 0;
  if (!full) return;
  const float L0k = pick<N>(tb.L[0], k), L1k = pick<N>(tb.L[1], k);
  float Dmk[N];
#pragma unroll
  for (int m = 0; m < N; ++m) Dmk[m] = pick<N>(tb.D[m], k);
  float dinv[M2], upp[M2];                  // this row of D'^{-1} and U of the previous cell
#pragma unroll
  for (int q = 0; q < M2; ++q) dinv[q] = upp[q] = 0.f;
  float alpha = 1.f;
  int eprev = -1;
  int e = head;
  for (int64_t j = 0; j < len && e >= 0; ++j) {
    const int ea = a.above[e];
    const int64_t nb = (int64_t)e * NP + t;
    float k22[N], hr[N];
#pragma unroll
    for (int m = 0; m < N; ++m) {
      k22[m] = (float)a.K[(int64_t)(DIM * DIM - 1) * Nn + nb + m * NFP];
      hr[m] = a.hscale * (float)a.plag[nb + m * NFP];
    }
    const float im = (float)a.invM[nb + k * NFP], ir = (float)a.irho[nb + k * NFP];
    if (j == 0) alpha = fmaxf(sqrtf(a.cd * hr[0] / (float)a.irho[nb]), 1.f);
    const float ia = 1.f / alpha;
    const int64_t sb = ((int64_t)e * NF + fb) * NFP + t, st = ((int64_t)e * NF + ftp) * NFP + t;
    const int kb = a.kind[sb], kt = a.kind[st];
    const bool cb = kb == 1 && eprev >= 0, ct = kt == 1 && ea >= 0;
    float nzb = a.nz[sb], nzt = a.nz[st];
    if (nzb == 0.f) nzb = -nzt;
    if (nzt == 0.f) nzt = -nzb;
    const float pcb = a.pc[sb], pct = a.pc[st];
    const float hmb = (float)a.trh[sb], hmt = (float)a.trh[st];
    const float hpb = cb ? (float)a.trh[((int64_t)eprev * NF + ftp) * NFP + t] : 0.f;
    const float hpt = ct ? (float)a.trh[((int64_t)ea * NF + fb) * NFP + t] : 0.f;
    const float wb = cb ? 0.5f : 1.f, wt = ct ? 0.5f : 1.f;
    float dg[M2], lo[M2], up[M2];
#pragma unroll
    for (int m = 0; m < N; ++m) {
      const float L0m = tb.L[0][m], L1m = tb.L[1][m];
      // vertical weak gradient G_z: volume term and central fluxes
      const float gs = im * (-Dmk[m] * k22[m] + wb * nzb * L0k * L0m + wt * nzt * L1k * L1m);
      const float gl = cb ? im * 0.5f * nzb * L0k * L1m : 0.f;
      const float gu = ct ? im * 0.5f * nzt * L1k * L0m : 0.f;
      if (xrow) {
        // vertical weak divergence of h rho w_z (no flux through walls)
        const float ds = im * (-Dmk[m] * hr[m] * k22[m] + (cb ? 0.5f * hmb * nzb * L0k * L0m : 0.f) +
                               (ct ? 0.5f * hmt * nzt * L1k * L1m : 0.f));
        const float dl = cb ? im * 0.5f * hpb * nzb * L0k * L1m : 0.f;
        const float du = ct ? im * 0.5f * hpt * nzt * L1k * L0m : 0.f;
        // penalty of the vertical faces
        const float ps = im * ((cb ? pcb * L0k * L0m : 0.f) + (ct ? pct * L1k * L1m : 0.f));
        const float pl = cb ? -im * pcb * L0k * L1m : 0.f;
        const float pu = ct ? -im * pct * L1k * L0m : 0.f;
        dg[m] = (k == m ? 1.f : 0.f) + ps - a.cg * gs;
        dg[N + m] = -a.cd * ds * ia;
        lo[m] = pl - a.cg * gl;
        lo[N + m] = -a.cd * dl * ia;
        up[m] = pu - a.cg * gu;
        up[N + m] = -a.cd * du * ia;
      } else {
        dg[m] = -alpha * ir * gs;
        dg[N + m] = k == m ? 1.f : 0.f;
        lo[m] = -alpha * ir * gl;
        lo[N + m] = 0.f;
        up[m] = -alpha * ir * gu;
        up[N + m] = 0.f;
      }
    }
    // mx = (L D'^{-1}_prev) row; dg -= (mx U_prev) row
    float mx[M2];
#pragma unroll
    for (int q = 0; q < M2; ++q) {
      float s = 0.f;
#pragma unroll
      for (int kk = 0; kk < M2; ++kk) s += lo[kk] * __shfl_sync(gmask, dinv[q], kk, G);
      mx[q] = j > 0 ? s : 0.f;
    }
#pragma unroll
    for (int q = 0; q < M2; ++q) {
      float s = 0.f;
#pragma unroll
      for (int kk = 0; kk < M2; ++kk) s += mx[kk] * __shfl_sync(gmask, upp[q], kk, G);
      dg[q] -= s;
    }
    // Gauss-Jordan inverse of the distributed rows, partial pivoting
    float x[M2];
#pragma unroll
    for (int q = 0; q < M2; ++q) x[q] = q == p ? 1.f : 0.f;
#pragma unroll
    for (int cc = 0; cc < M2; ++cc) {
      float v = (row && p >= cc) ? fabsf(dg[cc]) : -1.f;
      int vi = p;
#pragma unroll
      for (int off = G / 2; off > 0; off >>= 1) {
        const float ov = __shfl_xor_sync(gmask, v, off, G);
        const int oi = __shfl_xor_sync(gmask, vi, off, G);
        if (ov > v || (ov == v && oi < vi)) {
          v = ov;
          vi = oi;
        }
      }
      const int src = p == cc ? vi : (p == vi ? cc : p);
#pragma unroll
      for (int q = 0; q < M2; ++q) {
        dg[q] = __shfl_sync(gmask, dg[q], src, G);
        x[q] = __shfl_sync(gmask, x[q], src, G);
      }
      const float piv = __shfl_sync(gmask, dg[cc], cc, G);
      const float ip = piv != 0.f ? 1.f / piv : 0.f;
      if (p == cc) {
#pragma unroll
        for (int q = 0; q < M2; ++q) {
          dg[q] *= ip;
          x[q] *= ip;
        }
      }
      const float f = dg[cc];
#pragma unroll
      for (int q = 0; q < M2; ++q) {
        const float pa = __shfl_sync(gmask, dg[q], cc, G);
        const float px = __shfl_sync(gmask, x[q], cc, G);
        if (p != cc) {
          dg[q] -= f * pa;
          x[q] -= f * px;
        }
      }
    }
    if (row) {
      float* fo = a.fac + ((int64_t)e * NFP + t) * 3 * BS + p * M2;
#pragma unroll
      for (int q = 0; q < M2; q += 2) {
        reinterpret_cast<float2*>(fo)[q / 2] = make_float2(x[q], x[q + 1]);
        reinterpret_cast<float2*>(fo + BS)[q / 2] = make_float2(mx[q], mx[q + 1]);
        reinterpret_cast<float2*>(fo + 2 * BS)[q / 2] = make_float2(up[q], up[q + 1]);
      }
    }
#pragma unroll
    for (int q = 0; q < M2; ++q) {
      dinv[q] = x[q];
      upp[q] = up[q];
    }
    eprev = e;
    e = ea;
  }
}

// z = P^{-1} r: forward substitution up the chain, back substitution down.
// A group of G >= 2n threads per line, thread p owning row p of every block
// (rows >= 2n idle): its row of L Dinv_prev, U and Dinv is one contiguous
// load, the vector entries of the other rows come by shuffles in the group.
template <int DIM, int N>
__global__ void __launch_bounds__(256) k_vl_apply(VlArgs a, const double* __restrict__ r, double* __restrict__ z) {
  constexpr int NFP = ipow(N, DIM - 1), NP = ipow(N, DIM), M2 = 2 * N, BS = M2 * M2;
  constexpr int G = M2 <= 4 ? 4 : (M2 <= 8 ? 8 : 16);
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t line = gid / G;
  const int p = (int)(gid % G);
  if (line >= a.nchain * NFP) return;      // whole groups: G divides the block
  const int64_t c = line / NFP;
  const int t = (int)(line % NFP);
  const unsigned lane = threadIdx.x & 31u;
  const unsigned gmask = (G == 32 ? 0xffffffffu : ((1u << G) - 1u)) << (lane & ~(unsigned)(G - 1));
  const bool row = p < M2;
  const int pr = row ? p : 0;               // idle threads read row 0 and discard it
  const int head = a.heads[c];
  if (!a.vfull[c]) {
    int e = head;
    for (int64_t j = 0; j < a.E && e >= 0; ++j, e = a.above[e])
      if (p < N) {
        const int64_t node = (int64_t)e * NP + t + p * NFP;
        z[node] = r[node];
      }
    return;
  }
  float yp = 0.f;
  int e = head, tail = head;
  int64_t len = 0;
  for (; len < a.E && e >= 0; ++len) {
    const int64_t lc = (int64_t)e * NFP + t;
    float y = p < N ? (float)r[(int64_t)e * NP + t + p * NFP] : 0.f;
    if (len > 0) {
      float m[M2];
      load_row<M2>(a.fac + (lc * 3 + 1) * BS + pr * M2, m);
#pragma unroll
      for (int q = 0; q < M2; ++q) y -= m[q] * __shfl_sync(gmask, yp, q, G);
    }
    if (row) a.scr[lc * M2 + p] = y;
    yp = y;
    tail = e;
    e = a.above[e];
  }
  float zn = 0.f;
  e = tail;
  for (int64_t j = 0; j < len && e >= 0; ++j) {
    const int64_t lc = (int64_t)e * NFP + t;
    float y = row ? a.scr[lc * M2 + p] : 0.f;
    if (j > 0) {
      float u[M2];
      load_row<M2>(a.fac + (lc * 3 + 2) * BS + pr * M2, u);
#pragma unroll
      for (int q = 0; q < M2; ++q) y -= u[q] * __shfl_sync(gmask, zn, q, G);
    }
    float d[M2];
    load_row<M2>(a.fac + lc * 3 * BS + pr * M2, d);
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < M2; ++q) s += d[q] * __shfl_sync(gmask, y, q, G);
    if (p < N) z[(int64_t)e * NP + t + p * NFP] = (double)s;
    zn = s;
    e = a.below[e];
  }
}

VlArgs vl_args(dg_mesh* m) {
  const int64_t S = m->S;
  uint8_t* sb = m->vl_slots.as<uint8_t>();
  VlArgs a;
  a.above = m->vl_above;
  a.below = m->vl_below;
  a.heads = m->vl_heads;
  a.nchain = m->n_vchains;
  a.E = m->E;
  a.nz = reinterpret_cast<const float*>(sb);
  a.pc = reinterpret_cast<const float*>(sb + 4 * S);
  a.kind = reinterpret_cast<const int8_t*>(sb + 8 * S);
  a.vfull = sb + 9 * S;
  a.fac = m->vl_fac.as<float>();
  a.scr = m->vl_scr.as<float>();
  a.K = m->K;
  a.invM = m->invM;
  a.irho = m->irho.as<double>();
  a.trh = m->trh.as<double>();
  a.plag = nullptr;
  a.hscale = a.cd = a.cg = 0.f;
  return a;
}

template <int DIM, int N>
int vl_setup_impl(dg_mesh* m, const ImplK& k, const double* plag, int penalty, cudaStream_t st) {
  constexpr int M2 = 2 * N;
  const int64_t S = m->S, ES = m->E * m->nfp;
  int rc;
  if ((rc = m->vl_slots.ensure((size_t)9 * S + (size_t)m->n_vchains + 16)) != DG_OK) return rc;
  if ((rc = m->vl_fac.ensure(sizeof(float) * 3 * M2 * M2 * (size_t)ES)) != DG_OK) return rc;
  if ((rc = m->vl_scr.ensure(sizeof(float) * M2 * (size_t)ES)) != DG_OK) return rc;
  uint8_t* sb = m->vl_slots.as<uint8_t>();
  DG_CUDA(cudaMemsetAsync(sb, 0, (size_t)8 * S, st));
  DG_CUDA(cudaMemsetAsync(sb + 8 * S, 2, (size_t)S, st));
  VlArgs a = vl_args(m);
  if (m->nF > 0)
    DG_RUN(m, K_PRECOND_SETUP, st,
           k_vl_slots<<<grid_for(m->nF, 256), 256, 0, st>>>(topo(m), m->dim,
                                                             penalty ? m->pcoef.as<double>() : nullptr,
                                                             reinterpret_cast<float*>(sb),
                                                             reinterpret_cast<float*>(sb + 4 * S),
                                                             reinterpret_cast<int8_t*>(sb + 8 * S)));
  a.plag = plag;
  a.hscale = (float)(k.gamma / (k.gamma - 1.0));
  a.cd = (float)((k.gamma - 1.0) * k.a_dt * k.a_dt);
  a.cg = k.r2 ? (float)k.cgrav : 0.f;
  constexpr int G = M2 <= 4 ? 4 : (M2 <= 8 ? 8 : 16);
  const int64_t nth = m->n_vchains * m->nfp * G;
  if (nth > 0)
    DG_RUN(m, K_PRECOND_SETUP, st,
           (k_vl_setup<DIM, N><<<grid_for(nth, 256), 256, 0, st>>>(a, cast_tables<float>(m->tab.t))));
  DG_LAUNCH_CHECK("vertical-line setup");
  return DG_OK;
}

template <int DIM, int N>
int vl_apply_impl(dg_mesh* m, const double* r, double* z, cudaStream_t st) {
  VlArgs a = vl_args(m);
  constexpr int M2 = 2 * N, G = M2 <= 4 ? 4 : (M2 <= 8 ? 8 : 16);
  const int64_t nth = m->n_vchains * m->nfp * G;
  if (nth > 0) DG_RUN(m, K_PRECOND, st, (k_vl_apply<DIM, N><<<grid_for(nth, 256), 256, 0, st>>>(a, r, z)));
  DG_LAUNCH_CHECK("vertical-line apply");
  return DG_OK;
}

}  // namespace

int vline_setup(dg_mesh* m, const ImplK& k, const double* plag, int penalty, cudaStream_t st) {
  DG_DISPATCH(m, return (vl_setup_impl<D_, N_>(m, k, plag, penalty, st)));
  return DG_ERR_UNSUPPORTED;
}

int vline_apply(dg_mesh* m, const double* r, double* z, cudaStream_t st) {
  if (m->vl_fac.p == nullptr) {
    set_error("vertical-line preconditioner applied before its setup");
    return DG_ERR_ARG;
  }
  DG_DISPATCH(m, return (vl_apply_impl<D_, N_>(m, r, z, st)));
  return DG_ERR_UNSUPPORTED;
}

}  // namespace dg

using namespace dg;

extern "C" int dg_precond_apply(dg_ctx* ctx, const dg_mesh* mesh, const dg_phys* ph, const dg_implicit_coeffs* cf,
                                int precond, const double* r, double* z, void* stream) {
  if (!ctx || !mesh || !ph || !cf || !cf->rho || !cf->p_lag || !cf->u_lag || !r || !z || r == z) {
    set_error("dg_precond_apply: NULL or aliased argument");
    return DG_ERR_ARG;
  }
  if (!(ph->gamma > 1.0) || (ph->variant != DG_R1 && ph->variant != DG_R2)) {
    set_error("dg_precond_apply: invalid physics (gamma > 1, variant R1/R2)");
    return DG_ERR_ARG;
  }
  if (mesh->gll) {
    set_error("dg_precond_apply: the preconditioners are not implemented for Gauss-Lobatto nodes");
    return DG_ERR_UNSUPPORTED;
  }
  dg_mesh* m = const_cast<dg_mesh*>(mesh);
  cudaStream_t st = (cudaStream_t)stream;
  ImplK k = impl_consts(ph, cf->a_dt);
  int rc;
  if ((rc = prepare_rt(m, k, cf->rho, cf->p_lag, cf->u_lag, ph->penalty, st)) != DG_OK) return rc;
  if (precond != DG_PRECOND_VLINE && precond != DG_PRECOND_CELL) {
    set_error("dg_precond_apply: precond must be DG_PRECOND_VLINE or DG_PRECOND_CELL");
    return DG_ERR_ARG;
  }
  if ((rc = precond_setup(m, precond, k, cf->p_lag, ph->penalty, st)) != DG_OK) return rc;
  return precond_apply(m, r, z, st);
}
