// Cell-block (block-Jacobi) preconditioner of the scaled Schur system (not
// in the paper, whose GMRES runs unpreconditioned; meant for meshes whose
// stiff part the vertical lines do not reach, such as columns cut by 2:1
// faces).
//
// P is block diagonal with the exact diagonal blocks S_ee of the operator of
// Section 3.1, y = x + P_pen x - c_g G_z x - c_d Div(h rho w), w = rho^{-1}
// R G x (R = (I + beta J)^{-1} in R2, I in R1).  For x supported on cell e
// the block has two parts:
//  * the cell-local one: the weak gradient of x in e (volume term and the
//    own-trace half of the central face flux, or the whole wall value),
//    through rho^{-1} R, then the weak divergence in e (volume term and the
//    own half of the face flux, nothing through walls), gravity and the
//    penalty's own-trace term;
//  * the return through each conforming neighbour k: the face flux of x puts
//    a gradient into k along the normal lines of the face, and the
//    divergence's face flux brings it back, a term diagonal in the face
//    point t: c_d / 4 h_k(t) (n.R_k n)(t) sum_m l_m(face)^2 / (rho_k w det J_k)
//    along k's line through t, lifted into e by the trace weights.
// 2:1 faces keep only the cell-local half (their return terms need the
// prolongation and are left out).  The return through a neighbour comes back
// through the same face only when the neighbour touches the cell through one
// face; a periodic direction of 2 cells (both faces onto one neighbour) also
// has a return across to the opposite face, which the blocks leave out.  Each block (Np x Np, Np = (r+1)^d <= 64)
// is assembled and inverted by Gauss-Jordan with partial pivoting in shared
// memory, one block of threads per cell, in FP32; the solve is one FP32
// matrix-vector product per cell.
#include "solver.cuh"

namespace dg {

namespace {

// node of cell-local line `t` (tangential index) along direction a at
// position m (reference coordinates of the other directions from t)
template <int DIM, int N>
__device__ __forceinline__ int line_node(int a, int t, int m) {
  int idx[3] = {0, 0, 0};
  int r = t;
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    if (b == a) {
      idx[b] = m;
    } else {
      idx[b] = r % N;
      r /= N;
    }
  }
  return idx[0] + N * idx[1] + N * N * idx[2];
}

struct CbSlotArgs {
  const int* fp_minus;
  const int* fp_plus;
  const double* fgeo;      // (d + 1) x nF: n dS of the minus side
  const double* pcoef;     // nF, or null without the penalty
  const double* trh;       // S: traces of h rho
  const double* irho;      // N
  const double* invM;      // N
  const double* fcell;     // per-cell f, or null
  double f, a_dt, cd;
  int r2;
  int64_t nF, S, E;
  float* wg;               // S: own-trace weight of the gradient face flux
  float* wd;               // S: own-trace weight of the divergence face flux
  float* pc;               // S: penalty coefficient
  float* c2;               // S: return coefficient through the neighbour
};

__global__ void k_cb_prefill(int64_t S, float* wg, float* wd, float* pc, float* c2) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= S) return;
  wg[q] = 0.5f;      // coarse sides of 2:1 faces keep this own-trace half
  wd[q] = 0.5f;
  pc[q] = 0.f;
  c2[q] = 0.f;
}

template <int DIM, int N>
__device__ double return_factor(const CbSlotArgs& a, const Tables<double>& tb, int other, double n2h, double nz2) {
  constexpr int NFP = ipow(N, DIM - 1), NP = ipow(N, DIM), NF = 2 * DIM;
  const int64_t k = other / (NF * NFP);
  const int fo = (other / NFP) % NF, t = other % NFP;
  const int ao = fo / 2, so = fo % 2;
  double s = 0.0;
#pragma unroll
  for (int m = 0; m < N; ++m) {
    const int64_t node = k * NP + line_node<DIM, N>(ao, t, m);
    const double L = tb.L[so][m];
    s += L * L * a.irho[node] * a.invM[node];
  }
  double d = 1.0;
  if (a.r2) {
    const double beta = a.a_dt * (a.fcell ? a.fcell[k] : a.f);
    d = 1.0 / (1.0 + beta * beta);
  }
  // n.R n = d (horizontal part) + vertical part (the beta terms cancel)
  const double nrn = d * n2h + nz2;
  return 0.25 * a.cd * a.trh[other] * nrn * s;
}

// per face point: own-trace weights, penalty and return coefficients of both
// slots
template <int DIM, int N>
__global__ void k_cb_slots(CbSlotArgs a, Tables<double> tb) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= a.nF) return;
  const int sm = a.fp_minus[p], code = a.fp_plus[p];
  double n2h = 0.0, nz2 = 0.0;
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    const double v = a.fgeo[(int64_t)b * a.nF + p];
    if (b == DIM - 1) nz2 = v * v;
    else n2h += v * v;
  }
  const float pcv = a.pcoef ? (float)a.pcoef[p] : 0.f;
  if (code == -1) {
    a.wg[sm] = 1.f;
    a.wd[sm] = 0.f;
    a.pc[sm] = 0.f;
    a.c2[sm] = 0.f;
  } else if (code >= 0) {
    a.wg[sm] = a.wg[code] = 0.5f;
    a.wd[sm] = a.wd[code] = 0.5f;
    a.pc[sm] = a.pc[code] = pcv;
    a.c2[sm] = (float)return_factor<DIM, N>(a, tb, code, n2h, nz2);
    a.c2[code] = (float)return_factor<DIM, N>(a, tb, sm, n2h, nz2);
  } else {
    a.wg[sm] = 0.5f;
    a.wd[sm] = 0.5f;
    a.pc[sm] = pcv;
    a.c2[sm] = 0.f;
  }
}

struct CbAsmArgs {
  int64_t E, S;
  int terrain, r2;
  const double* K;        // d*d x N
  const double* invM;     // N
  const double* irho;     // N
  const double* plag;     // N
  const double* trh;      // S
  const double* nS;       // d x S: outward n dS per slot
  const float* wg;
  const float* wd;
  const float* pc;
  const float* c2;
  const double* fcell;
  double f, a_dt;
  float hscale, cd, cg;
  float* inv;             // E x Np x Np, column-major per cell
};

template <int DIM, int N>
struct CbShape {
  static constexpr int NP = ipow(N, DIM), NFP = ipow(N, DIM - 1), NS = 2 * DIM * NFP;
  static constexpr int WS = NP * DIM + 1;          // column stride of W (padded)
  static constexpr int AS = 2 * NP + 1;            // row stride of A (padded)
  static constexpr int SDW = DIM + 5;              // floats per slot record
  static constexpr int FLOATS = NP * WS + NP * AS + DIM * DIM * NP + 3 * NP + N * N + 2 * N + NS * SDW + 4;
  static constexpr size_t BYTES = sizeof(float) * FLOATS;
};

// One block of NP threads per cell: thread j builds column j of the gradient
// (through rho^{-1} R), thread i row i of the block, then Gauss-Jordan.
template <int DIM, int N>
__global__ void k_cb_assemble(CbAsmArgs g, Tables<float> tb) {
  using CB = CbShape<DIM, N>;
  constexpr int NP = CB::NP, NFP = CB::NFP, NS = CB::NS, WS = CB::WS, AS = CB::AS, SDW = CB::SDW;
  extern __shared__ float sh[];
  float* W = sh;                        // W[j * WS + m * DIM + b]
  float* A = W + NP * WS;               // A[i * AS + c]
  float* Kn = A + NP * AS;              // Kn[(a * DIM + b) * NP + m]
  float* iMs = Kn + DIM * DIM * NP;
  float* irs = iMs + NP;
  float* hrs = irs + NP;
  float* Dt = hrs + NP;                 // D[k][j] = l_j'(xi_k)
  float* Lt = Dt + N * N;               // L[s][j]
  float* SD = Lt + 2 * N;               // per slot: nS[DIM], wg, wd, pc, c2, h
  float* cst = SD + NS * SDW;           // beta, d
  __shared__ int piv_s;
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x;
  const int64_t Nn = g.E * NP;
  const int64_t node = e * NP + tid;
#pragma unroll
  for (int a = 0; a < DIM; ++a)
#pragma unroll
    for (int b = 0; b < DIM; ++b)
      Kn[(a * DIM + b) * NP + tid] =
          (g.terrain && kzero<DIM>(a, b)) ? 0.f : (float)g.K[(int64_t)(a * DIM + b) * Nn + node];
  iMs[tid] = (float)g.invM[node];
  irs[tid] = (float)g.irho[node];
  hrs[tid] = g.hscale * (float)g.plag[node];
  if (tid == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
#pragma unroll
      for (int j = 0; j < N; ++j) Dt[k * N + j] = tb.D[k][j];
      Lt[k] = tb.L[0][k];
      Lt[N + k] = tb.L[1][k];
    }
    double d = 1.0, beta = 0.0;
    if (g.r2) {
      beta = g.a_dt * (g.fcell ? g.fcell[e] : g.f);
      d = 1.0 / (1.0 + beta * beta);
    }
    cst[0] = (float)beta;
    cst[1] = (float)d;
  }
  for (int q = tid; q < NS; q += NP) {
    const int64_t slot = e * NS + q;
#pragma unroll
    for (int b = 0; b < DIM; ++b) SD[q * SDW + b] = (float)g.nS[(int64_t)b * g.S + slot];
    SD[q * SDW + DIM] = g.wg[slot];
    SD[q * SDW + DIM + 1] = g.wd[slot];
    SD[q * SDW + DIM + 2] = g.pc[slot];
    SD[q * SDW + DIM + 3] = g.c2[slot];
    SD[q * SDW + DIM + 4] = (float)g.trh[slot];
  }
  __syncthreads();
  // ---- column j: w = rho^{-1} R G e_j at every node of the cell
  {
    const int j = tid;
    int idj[3];
    node_index<DIM, N>(j, idj);
    float* Wj = W + j * WS;
    for (int q = 0; q < NP * DIM; ++q) Wj[q] = 0.f;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int stride = a == 0 ? 1 : (a == 1 ? N : N * N);
      const int base = j - idj[a] * stride;
      // volume: -D[idx_a(j)][idx_a(m)] K_ab(j) along the a-line through j
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const int mm = base + k * stride;
        const float dk = Dt[idj[a] * N + k];
#pragma unroll
        for (int b = 0; b < DIM; ++b) Wj[mm * DIM + b] -= dk * Kn[(a * DIM + b) * NP + j];
      }
      // faces: own-trace part of the flux, lifted along the same line
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int q = (2 * a + s) * NFP + tang_index<DIM, N>(idj, a);
        const float avg = SD[q * SDW + DIM] * Lt[s * N + idj[a]];
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const int mm = base + k * stride;
#pragma unroll
          for (int b = 0; b < DIM; ++b) Wj[mm * DIM + b] += avg * SD[q * SDW + b] * Lt[s * N + k];
        }
      }
    }
    const float beta = cst[0], d = cst[1];
    for (int mm = 0; mm < NP; ++mm) {
      float G[DIM];
#pragma unroll
      for (int b = 0; b < DIM; ++b) G[b] = iMs[mm] * Wj[mm * DIM + b];
      const float ir = irs[mm];
      if (DIM == 3) {
        Wj[mm * DIM + 0] = g.r2 ? (G[0] + beta * G[1]) * d * ir : G[0] * ir;
        Wj[mm * DIM + 1] = g.r2 ? (G[1] - beta * G[0]) * d * ir : G[1] * ir;
        Wj[mm * DIM + DIM - 1] = G[DIM - 1] * ir;
      } else {
        Wj[mm * DIM + 0] = g.r2 ? G[0] * d * ir : G[0] * ir;
        Wj[mm * DIM + DIM - 1] = G[DIM - 1] * ir;
      }
    }
  }
  __syncthreads();
  // ---- row i of the block
  {
    const int i = tid;
    int idi[3];
    node_index<DIM, N>(i, idi);
    float* Ai = A + i * AS;
    for (int j = 0; j < NP; ++j) {
      const float* Wj = W + j * WS;
      int idj[3];
      node_index<DIM, N>(j, idj);
      float acc = 0.f, self = 0.f;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const int stride = a == 0 ? 1 : (a == 1 ? N : N * N);
        const int base = i - idi[a] * stride;
        // volume: sum_k D[k][idx_a(i)] (-h rho_m sum_b K_ab(m) w_b(m))
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const int mm = base + k * stride;
          float v = 0.f;
#pragma unroll
          for (int b = 0; b < DIM; ++b) v += Kn[(a * DIM + b) * NP + mm] * Wj[mm * DIM + b];
          acc -= Dt[k * N + idi[a]] * hrs[mm] * v;
        }
        const bool online = tang_index<DIM, N>(idi, a) == tang_index<DIM, N>(idj, a);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const int q = (2 * a + s) * NFP + tang_index<DIM, N>(idi, a);
          float wtr = 0.f;
#pragma unroll
          for (int k = 0; k < N; ++k) {
            const int mm = base + k * stride;
            float wn = 0.f;
#pragma unroll
            for (int b = 0; b < DIM; ++b) wn += Wj[mm * DIM + b] * SD[q * SDW + b];
            wtr += Lt[s * N + k] * wn;
          }
          const float Li = Lt[s * N + idi[a]];
          acc += SD[q * SDW + DIM + 1] * SD[q * SDW + DIM + 4] * wtr * Li;
          if (online) self += Li * Lt[s * N + idj[a]] * (SD[q * SDW + DIM + 2] + SD[q * SDW + DIM + 3]);
        }
      }
      // G_z(i) = w_z(i) / (1/rho): the vertical component is not rotated
      const float gz = Wj[i * DIM + DIM - 1] / irs[i];
      Ai[j] = (i == j ? 1.f : 0.f) + iMs[i] * self - g.cd * iMs[i] * acc - g.cg * gz;
      Ai[NP + j] = i == j ? 1.f : 0.f;
    }
  }
  __syncthreads();
  // ---- Gauss-Jordan with partial pivoting on [S_ee | I]
  for (int c = 0; c < NP; ++c) {
    if (tid == 0) {
      int pv = c;
      float best = fabsf(A[c * AS + c]);
      for (int r = c + 1; r < NP; ++r) {
        const float v = fabsf(A[r * AS + c]);
        if (v > best) {
          best = v;
          pv = r;
        }
      }
      piv_s = pv;
    }
    __syncthreads();
    const int pv = piv_s;
    if (pv != c)
      for (int col = tid; col < 2 * NP; col += NP) {
        const float t = A[c * AS + col];
        A[c * AS + col] = A[pv * AS + col];
        A[pv * AS + col] = t;
      }
    __syncthreads();
    const float pivot = A[c * AS + c];
    const float ip = pivot != 0.f ? 1.f / pivot : 0.f;
    __syncthreads();
    for (int col = tid; col < 2 * NP; col += NP) A[c * AS + col] *= ip;
    __syncthreads();
    if (tid != c) {
      const float fct = A[tid * AS + c];
      if (fct != 0.f)
        for (int col = 0; col < 2 * NP; ++col) A[tid * AS + col] -= fct * A[c * AS + col];
    }
    __syncthreads();
  }
  // inverse, column-major per cell: inv[(e NP + j) NP + i]
  float* out = g.inv + e * (int64_t)NP * NP;
  for (int j = 0; j < NP; ++j) out[j * NP + tid] = A[tid * AS + NP + j];
}

// z_e = S_ee^{-1} r_e, several cells per block
template <int DIM, int N>
__global__ void __launch_bounds__(256) k_cb_apply(const float* __restrict__ inv, const double* __restrict__ r,
                                                  double* __restrict__ z, int64_t E) {
  constexpr int NP = ipow(N, DIM), EPB = NP >= 256 ? 1 : 256 / NP;
  __shared__ float rs[EPB][NP];
  const int le = threadIdx.x / NP, i = threadIdx.x % NP;
  const int64_t e = (int64_t)blockIdx.x * EPB + le;
  const bool active = e < E;
  rs[le][i] = active ? (float)r[e * NP + i] : 0.f;
  __syncthreads();
  if (!active) return;
  const float* P = inv + e * (int64_t)NP * NP;
  float acc = 0.f;
#pragma unroll 8
  for (int j = 0; j < NP; ++j) acc += __ldg(P + j * NP + i) * rs[le][j];
  z[e * NP + i] = (double)acc;
}

template <int DIM, int N>
int cb_setup_impl(dg_mesh* m, const ImplK& k, const double* plag, int penalty, cudaStream_t st) {
  using CB = CbShape<DIM, N>;
  constexpr int NP = CB::NP;
  if (DIM == 3 && N > 4) {
    set_error("cell-block preconditioner: blocks of (r+1)^3 > 64 nodes are not supported (3D degree <= 3)");
    return DG_ERR_UNSUPPORTED;
  }
  const int64_t S = m->S, E = m->E;
  int rc;
  if ((rc = m->cb_slots.ensure(sizeof(double) * DIM * S + sizeof(float) * 4 * S + 64)) != DG_OK) return rc;
  if ((rc = m->cb_inv.ensure(sizeof(float) * (size_t)E * NP * NP)) != DG_OK) return rc;
  double* nS = m->cb_slots.as<double>();
  float* fl = reinterpret_cast<float*>(nS + (size_t)DIM * S);
  float *wg = fl, *wd = fl + S, *pc = fl + 2 * S, *c2 = fl + 3 * S;
  if ((rc = slot_normals(m, nS, st)) != DG_OK) return rc;
  DG_RUN(m, K_PRECOND_SETUP, st, k_cb_prefill<<<grid_for(S, 256), 256, 0, st>>>(S, wg, wd, pc, c2));
  CbSlotArgs sa;
  sa.fp_minus = m->fp_minus;
  sa.fp_plus = m->fp_plus;
  sa.fgeo = m->fgeo;
  sa.pcoef = penalty ? m->pcoef.as<double>() : nullptr;
  sa.trh = m->trh.as<double>();
  sa.irho = m->irho.as<double>();
  sa.invM = m->invM;
  sa.fcell = k.fcell;
  sa.f = k.f;
  sa.a_dt = k.a_dt;
  sa.cd = (k.gamma - 1.0) * k.a_dt * k.a_dt;
  sa.r2 = k.r2;
  sa.nF = m->nF;
  sa.S = S;
  sa.E = E;
  sa.wg = wg;
  sa.wd = wd;
  sa.pc = pc;
  sa.c2 = c2;
  if (m->nF > 0)
    DG_RUN(m, K_PRECOND_SETUP, st, (k_cb_slots<DIM, N><<<grid_for(m->nF, 256), 256, 0, st>>>(sa, m->tab.t)));
  CbAsmArgs g;
  g.E = E;
  g.S = S;
  g.terrain = m->terrain ? 1 : 0;
  g.r2 = k.r2;
  g.K = m->K;
  g.invM = m->invM;
  g.irho = m->irho.as<double>();
  g.plag = plag;
  g.trh = m->trh.as<double>();
  g.nS = nS;
  g.wg = wg;
  g.wd = wd;
  g.pc = pc;
  g.c2 = c2;
  g.fcell = k.fcell;
  g.f = k.f;
  g.a_dt = k.a_dt;
  g.hscale = (float)(k.gamma / (k.gamma - 1.0));
  g.cd = (float)((k.gamma - 1.0) * k.a_dt * k.a_dt);
  g.cg = k.r2 ? (float)k.cgrav : 0.f;
  g.inv = m->cb_inv.as<float>();
  static bool attr_set = false;   // per (DIM, N) instantiation
  if (!attr_set) {
    DG_CUDA(cudaFuncSetAttribute(k_cb_assemble<DIM, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)CB::BYTES));
    attr_set = true;
  }
  if (E > 0)
    DG_RUN(m, K_PRECOND_SETUP, st,
           (k_cb_assemble<DIM, N><<<(unsigned)E, NP, CB::BYTES, st>>>(g, cast_tables<float>(m->tab.t))));
  DG_LAUNCH_CHECK("cell-block setup");
  m->pc_kind = DG_PRECOND_CELL;
  return DG_OK;
}

template <int DIM, int N>
int cb_apply_impl(dg_mesh* m, const double* r, double* z, cudaStream_t st) {
  constexpr int NP = ipow(N, DIM), EPB = NP >= 256 ? 1 : 256 / NP;
  if (m->E > 0)
    DG_RUN(m, K_PRECOND, st,
           (k_cb_apply<DIM, N><<<grid_for(m->E, EPB), EPB * NP, 0, st>>>(m->cb_inv.as<float>(), r, z, m->E)));
  DG_LAUNCH_CHECK("cell-block apply");
  return DG_OK;
}

}  // namespace

int cellblock_setup(dg_mesh* m, const ImplK& k, const double* plag, int penalty, cudaStream_t st) {
  DG_DISPATCH(m, return (cb_setup_impl<D_, N_>(m, k, plag, penalty, st)));
  return DG_ERR_UNSUPPORTED;
}

int cellblock_apply(dg_mesh* m, const double* r, double* z, cudaStream_t st) {
  if (m->cb_inv.p == nullptr) {
    set_error("cell-block preconditioner applied before its setup");
    return DG_ERR_ARG;
  }
  DG_DISPATCH(m, return (cb_apply_impl<D_, N_>(m, r, z, st)));
  return DG_ERR_UNSUPPORTED;
}

int precond_setup(dg_mesh* m, int kind, const ImplK& k, const double* plag, int penalty, cudaStream_t st) {
  if (kind == DG_PRECOND_VLINE) {
    const int rc = vline_setup(m, k, plag, penalty, st);
    if (rc == DG_OK) m->pc_kind = DG_PRECOND_VLINE;
    return rc;
  }
  if (kind == DG_PRECOND_CELL) return cellblock_setup(m, k, plag, penalty, st);
  set_error("unknown preconditioner %d", kind);
  return DG_ERR_ARG;
}

int precond_apply(dg_mesh* m, const double* r, double* z, cudaStream_t st) {
  if (m->pc_kind == DG_PRECOND_VLINE) return vline_apply(m, r, z, st);
  if (m->pc_kind == DG_PRECOND_CELL) return cellblock_apply(m, r, z, st);
  set_error("preconditioner applied before its setup");
  return DG_ERR_ARG;
}

}  // namespace dg
