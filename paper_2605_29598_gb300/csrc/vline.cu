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
// pivoting), one thread per line.  The unknown w_z is carried as alpha w_z,
// alpha = sqrt(c_d h rho rho) at the line's first node, which balances the
// x-w and w-x couplings (their entries differ by ~1e7 otherwise, and the
// unscaled 2n x 2n blocks lose most FP32 digits).  Only chains that end in walls at both
// ends are factored; the lines of other chains (cut by a 2:1 face, or a
// vertically periodic column) are left unpreconditioned (identity).
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

template <int M>
__device__ __forceinline__ void mat_mul(const float (&A)[M][M], const float (&B)[M][M], float (&C)[M][M]) {
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) {
      float s = 0.f;
      for (int k = 0; k < M; ++k) s += A[i][k] * B[k][j];
      C[i][j] = s;
    }
}

// Gauss-Jordan inverse with partial pivoting (A is destroyed)
template <int M>
__device__ __forceinline__ void mat_inv(float (&A)[M][M], float (&X)[M][M]) {
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) X[i][j] = i == j ? 1.f : 0.f;
  for (int c = 0; c < M; ++c) {
    int piv = c;
    float best = fabsf(A[c][c]);
    for (int i = c + 1; i < M; ++i)
      if (fabsf(A[i][c]) > best) {
        best = fabsf(A[i][c]);
        piv = i;
      }
    if (piv != c)
      for (int j = 0; j < M; ++j) {
        float t = A[c][j];
        A[c][j] = A[piv][j];
        A[piv][j] = t;
        t = X[c][j];
        X[c][j] = X[piv][j];
        X[piv][j] = t;
      }
    const float ip = best > 0.f ? 1.f / A[c][c] : 0.f;
    for (int j = 0; j < M; ++j) {
      A[c][j] *= ip;
      X[c][j] *= ip;
    }
    for (int i = 0; i < M; ++i) {
      if (i == c) continue;
      const float f = A[i][c];
      if (f == 0.f) continue;
      for (int j = 0; j < M; ++j) {
        A[i][j] -= f * A[c][j];
        X[i][j] -= f * X[c][j];
      }
    }
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
  float* fac;              // 3 blocks (Dinv, L Dinv_prev, U) x (2n)^2 entries x E nfp
  float* scr;              // 2n x E nfp
  const double* K;         // d*d x N metric (K_dd used)
  const double* invM;      // N
  const double* irho;      // N
  const double* trh;       // S : traces of h rho = gamma p_lag / (gamma - 1)
  const double* plag;      // N
  float hscale, cd, cg;    // gamma/(gamma-1), (gamma-1) a_dt^2, (gamma-1) a_dt^2 g (R2) or 0
};

// One thread per (chain, horizontal node position t): assembles the three
// 2n x 2n blocks of every cell of the line and runs the forward sweep of
// block Thomas, storing D'^{-1}, L D'^{-1}_prev and U per cell.
template <int DIM, int N>
__global__ void __launch_bounds__(128) k_vl_setup(VlArgs a, Tables<float> tb) {
  constexpr int NFP = ipow(N, DIM - 1), NP = ipow(N, DIM), NF = 2 * DIM, M2 = 2 * N, BS = M2 * M2;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= a.nchain * NFP) return;
  const int64_t c = gid / NFP;
  const int t = (int)(gid % NFP);
  const int fb = 2 * (DIM - 1), ftp = fb + 1;
  const int64_t ES = a.E * NFP, Nn = a.E * NP;
  const int head = a.heads[c];
  int tail = head;
  int64_t len = 1;
  while (a.above[tail] >= 0 && len < a.E) {
    tail = a.above[tail];
    ++len;
  }
  const bool full = a.kind[((int64_t)head * NF + fb) * NFP + t] == 0 &&
                    a.kind[((int64_t)tail * NF + ftp) * NFP + t] == 0;
  if (t == 0) a.vfull[c] = full ? 1 : 0;
  if (!full) return;
  float Dinv[M2][M2], Upp[M2][M2];
  float alpha = 1.f;
  int eprev = -1;
  int e = head;
  for (int64_t j = 0; j < len && e >= 0; ++j) {
    const int ea = a.above[e];
    float k22[N], im[N], ir[N], hr[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int64_t node = (int64_t)e * NP + t + k * NFP;
      k22[k] = (float)a.K[(int64_t)(DIM * DIM - 1) * Nn + node];
      im[k] = (float)a.invM[node];
      ir[k] = (float)a.irho[node];
      hr[k] = a.hscale * (float)a.plag[node];
    }
    if (j == 0) alpha = fmaxf(sqrtf(a.cd * hr[0] / ir[0]), 1.f);
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
    float Dg[M2][M2], Lo[M2][M2], Up[M2][M2];
    for (int k = 0; k < N; ++k) {
      const float L0k = tb.L[0][k], L1k = tb.L[1][k];
      for (int m = 0; m < N; ++m) {
        const float L0m = tb.L[0][m], L1m = tb.L[1][m];
        // vertical weak gradient G_z: volume term and central fluxes
        const float gs = im[k] * (-tb.D[m][k] * k22[m] + wb * nzb * L0k * L0m + wt * nzt * L1k * L1m);
        const float gl = cb ? im[k] * 0.5f * nzb * L0k * L1m : 0.f;
        const float gu = ct ? im[k] * 0.5f * nzt * L1k * L0m : 0.f;
        // vertical weak divergence of h rho w_z (no flux through walls)
        const float ds = im[k] * (-tb.D[m][k] * hr[m] * k22[m] + (cb ? 0.5f * hmb * nzb * L0k * L0m : 0.f) +
                                  (ct ? 0.5f * hmt * nzt * L1k * L1m : 0.f));
        const float dl = cb ? im[k] * 0.5f * hpb * nzb * L0k * L1m : 0.f;
        const float du = ct ? im[k] * 0.5f * hpt * nzt * L1k * L0m : 0.f;
        // penalty of the vertical faces
        const float ps = im[k] * ((cb ? pcb * L0k * L0m : 0.f) + (ct ? pct * L1k * L1m : 0.f));
        const float pl = cb ? -im[k] * pcb * L0k * L1m : 0.f;
        const float pu = ct ? -im[k] * pct * L1k * L0m : 0.f;
        Dg[k][m] = (k == m ? 1.f : 0.f) + ps - a.cg * gs;
        Dg[k][N + m] = -a.cd * ds * ia;
        Dg[N + k][m] = -alpha * ir[k] * gs;
        Dg[N + k][N + m] = k == m ? 1.f : 0.f;
        Lo[k][m] = pl - a.cg * gl;
        Lo[k][N + m] = -a.cd * dl * ia;
        Lo[N + k][m] = -alpha * ir[k] * gl;
        Lo[N + k][N + m] = 0.f;
        Up[k][m] = pu - a.cg * gu;
        Up[k][N + m] = -a.cd * du * ia;
        Up[N + k][m] = -alpha * ir[k] * gu;
        Up[N + k][N + m] = 0.f;
      }
    }
    float Mx[M2][M2];
    if (j == 0) {
      for (int p = 0; p < M2; ++p)
        for (int q = 0; q < M2; ++q) Mx[p][q] = 0.f;
    } else {
      mat_mul<M2>(Lo, Dinv, Mx);
      mat_mul<M2>(Mx, Upp, Lo);      // Lo <- L D'^{-1}_prev U_prev
      for (int p = 0; p < M2; ++p)
        for (int q = 0; q < M2; ++q) Dg[p][q] -= Lo[p][q];
    }
    mat_inv<M2>(Dg, Dinv);
    const int64_t base = (int64_t)e * NFP + t;
    for (int p = 0; p < M2; ++p)
      for (int q = 0; q < M2; ++q) {
        const int64_t ent = p * M2 + q;
        a.fac[ent * ES + base] = Dinv[p][q];
        a.fac[(BS + ent) * ES + base] = Mx[p][q];
        a.fac[(2 * BS + ent) * ES + base] = Up[p][q];
        Upp[p][q] = Up[p][q];
      }
    eprev = e;
    e = ea;
  }
}

// z = P^{-1} r: forward substitution up the chain, back substitution down
template <int DIM, int N>
__global__ void __launch_bounds__(128) k_vl_apply(VlArgs a, const double* __restrict__ r, double* __restrict__ z) {
  constexpr int NFP = ipow(N, DIM - 1), NP = ipow(N, DIM), M2 = 2 * N, BS = M2 * M2;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= a.nchain * NFP) return;
  const int64_t c = gid / NFP;
  const int t = (int)(gid % NFP);
  const int64_t ES = a.E * NFP;
  const int head = a.heads[c];
  if (!a.vfull[c]) {
    int e = head;
    for (int64_t j = 0; j < a.E && e >= 0; ++j, e = a.above[e])
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const int64_t node = (int64_t)e * NP + t + k * NFP;
        z[node] = r[node];
      }
    return;
  }
  float yp[M2];
  int e = head, tail = head;
  int64_t len = 0;
  for (; len < a.E && e >= 0; ++len) {
    const int64_t base = (int64_t)e * NFP + t;
    float y[M2];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      y[k] = (float)r[(int64_t)e * NP + t + k * NFP];
      y[N + k] = 0.f;
    }
    if (len > 0) {
#pragma unroll
      for (int p = 0; p < M2; ++p) {
        float s = y[p];
#pragma unroll
        for (int q = 0; q < M2; ++q) s -= a.fac[(BS + p * M2 + q) * ES + base] * yp[q];
        y[p] = s;
      }
    }
#pragma unroll
    for (int p = 0; p < M2; ++p) {
      a.scr[p * ES + base] = y[p];
      yp[p] = y[p];
    }
    tail = e;
    e = a.above[e];
  }
  float zn[M2];
  e = tail;
  for (int64_t j = 0; j < len && e >= 0; ++j) {
    const int64_t base = (int64_t)e * NFP + t;
    float y[M2];
#pragma unroll
    for (int p = 0; p < M2; ++p) y[p] = a.scr[p * ES + base];
    if (j > 0) {
#pragma unroll
      for (int p = 0; p < M2; ++p) {
        float s = y[p];
#pragma unroll
        for (int q = 0; q < M2; ++q) s -= a.fac[(2 * BS + p * M2 + q) * ES + base] * zn[q];
        y[p] = s;
      }
    }
    float zz[M2];
#pragma unroll
    for (int p = 0; p < M2; ++p) {
      float s = 0.f;
#pragma unroll
      for (int q = 0; q < M2; ++q) s += a.fac[(p * M2 + q) * ES + base] * y[q];
      zz[p] = s;
    }
#pragma unroll
    for (int k = 0; k < N; ++k) z[(int64_t)e * NP + t + k * NFP] = (double)zz[k];
#pragma unroll
    for (int p = 0; p < M2; ++p) zn[p] = zz[p];
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
    DG_RUN(m, K_VLINE_SETUP, st,
           k_vl_slots<<<grid_for(m->nF, 256), 256, 0, st>>>(topo(m), m->dim,
                                                             penalty ? m->pcoef.as<double>() : nullptr,
                                                             reinterpret_cast<float*>(sb),
                                                             reinterpret_cast<float*>(sb + 4 * S),
                                                             reinterpret_cast<int8_t*>(sb + 8 * S)));
  a.plag = plag;
  a.hscale = (float)(k.gamma / (k.gamma - 1.0));
  a.cd = (float)((k.gamma - 1.0) * k.a_dt * k.a_dt);
  a.cg = k.r2 ? (float)k.cgrav : 0.f;
  const int64_t nth = m->n_vchains * m->nfp;
  if (nth > 0)
    DG_RUN(m, K_VLINE_SETUP, st,
           (k_vl_setup<DIM, N><<<grid_for(nth, 128), 128, 0, st>>>(a, cast_tables<float>(m->tab.t))));
  DG_LAUNCH_CHECK("vertical-line setup");
  return DG_OK;
}

template <int DIM, int N>
int vl_apply_impl(dg_mesh* m, const double* r, double* z, cudaStream_t st) {
  VlArgs a = vl_args(m);
  const int64_t nth = m->n_vchains * m->nfp;
  if (nth > 0) DG_RUN(m, K_VLINE, st, (k_vl_apply<DIM, N><<<grid_for(nth, 128), 128, 0, st>>>(a, r, z)));
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
                                const double* r, double* z, void* stream) {
  if (!ctx || !mesh || !ph || !cf || !cf->rho || !cf->p_lag || !cf->u_lag || !r || !z || r == z) {
    set_error("dg_precond_apply: NULL or aliased argument");
    return DG_ERR_ARG;
  }
  if (!(ph->gamma > 1.0) || (ph->variant != DG_R1 && ph->variant != DG_R2)) {
    set_error("dg_precond_apply: invalid physics (gamma > 1, variant R1/R2)");
    return DG_ERR_ARG;
  }
  dg_mesh* m = const_cast<dg_mesh*>(mesh);
  cudaStream_t st = (cudaStream_t)stream;
  ImplK k = impl_consts(ph, cf->a_dt);
  int rc;
  if ((rc = prepare_rt(m, k, cf->rho, cf->p_lag, cf->u_lag, ph->penalty, st)) != DG_OK) return rc;
  if ((rc = vline_setup(m, k, cf->p_lag, ph->penalty, st)) != DG_OK) return rc;
  return vline_apply(m, r, z, st);
}
