// Discrete adjoint of the stream-collide step, the mean-flux objective and the
// sqrt(T) checkpointed forward/backward driver.
//
// The paper has no adjoint.  The forward map whose transpose is taken here is
// the step of Eq. 1 with the TRT collision (Sect. 2) and pull streaming
// (Sect. 4): F_{n+1} = S(C(F_n; s)).  With lambda_{n+1} = dJ/dF_{n+1}:
//   mu            = S^T lambda_{n+1}   (gather through the mirrored direction)
//   lambda_n      = (dC/dF)^T mu,   grad_s += (dC/ds)^T mu.
// Writing C_i = f_i - l+ f+_i - l- f-_i + G_i(rho, u, s) with
// G_i = l+ feq+_i + l- feq-_i + a+ S+_i + a- S-_i, the transpose of the
// linear part is symmetric, and sum_i mu_i G_i = rho Psi(u, s) depends on mu
// only through M0 = sum w mu, M1 = sum w c mu, M2 = sum w c c^T mu:
//   Psi = l+ M0 (1 - 3/2 u.u) + 9/2 l+ q + 3 l- a + 9 a+ u.M2 g - 9 a+ s q
//         - 3 a+ M0 u.g + 3 a+ M0 s u.u + 3 a- M1.g - 3 a- s a,
//   q = u.M2 u, a = M1.u.
// Then, with u = kd (j0/rho + g/2), kd = 1/(1 + s/2):
//   lambda_n[k] = mu_k - l+ mu+_k - l- mu-_k + A + B.c_k,
//   A = Psi - dPsi/du . (u - kd g/2),  B = kd dPsi/du,
//   grad_s += rho (dPsi/ds - kd/2 dPsi/du . u).
#include "kernels.cuh"

namespace lbm {
namespace dev {

template <class R> struct AdjConst {
  R lp, lm, ap, am;  // l+, l-, a+ = 1 - l+/2, a- = 1 - l-/2
  R qp, qm;          // (1 - l+)/2, (1 - l-)/2
  R g[3], hg[3];
  R rho_s;
  R w[3];            // D3Q19 weights 1/3, 1/18, 1/36
  R omlp;            // 1 - l+
};

// Storage of the adjoint arrays: IEEE double for both FP64 paths (the
// double-float one converts on load and store), float otherwise.
template <int PREC> struct Lam {
  using T = float;
  static __device__ __forceinline__ float ld(const T* p) { return *p; }
  static __device__ __forceinline__ void st(T* p, float v) { *p = v; }
  static __device__ __forceinline__ double to_double(float v) { return double(v); }
};
template <> struct Lam<LBM_F64> {
  using T = double;
  static __device__ __forceinline__ double ld(const T* p) { return *p; }
  static __device__ __forceinline__ void st(T* p, double v) { *p = v; }
  static __device__ __forceinline__ double to_double(double v) { return v; }
};
template <> struct Lam<LBM_F64_DF> {
  using T = double;
  static __device__ __forceinline__ df ld(const T* p) { return df_from_double(*p); }
  static __device__ __forceinline__ void st(T* p, df v) { *p = double_from_df(v); }
  static __device__ __forceinline__ double to_double(df v) { return double_from_df(v); }
};

template <class R> AdjConst<R> make_adj(const KParams& kp) {
  AdjConst<R> c;
  c.w[0] = R(1.0 / 3.0);
  c.w[1] = R(1.0 / 18.0);
  c.w[2] = R(1.0 / 36.0);
  c.omlp = R(1.0 - kp.lp);
  c.lp = R(kp.lp);
  c.lm = R(kp.lm);
  c.ap = R(1.0 - kp.lp / 2);
  c.am = R(1.0 - kp.lm / 2);
  c.qp = R((1.0 - kp.lp) / 2);
  c.qm = R((1.0 - kp.lm) / 2);
  for (int a = 0; a < 3; ++a) {
    c.g[a] = R(kp.g[a]);
    c.hg[a] = R(kp.g[a] / 2);
  }
  c.rho_s = R(kp.rho_s);
  return c;
}

// One adjoint step.  G: OS-NT grid at step n (its pull gather is F_n).
// lam_next / lam: adjoint of the canonical states F_{n+1} / F_n, layout [19][Npad].
template <int PREC, bool RIA, bool DRAG>
__global__ void __launch_bounds__(kBlock) k_adjoint(DevTables t, KParams kp, CollConst<typename St<PREC>::R> cc,
                                                    AdjConst<typename St<PREC>::R> c,
                                                    const typename St<PREC>::T* __restrict__ G,
                                                    const typename Lam<PREC>::T* __restrict__ lam_next,
                                                    typename Lam<PREC>::T* __restrict__ lam,
                                                    const float* __restrict__ s, double* __restrict__ grad_s, int N) {
  using R = typename St<PREC>::R;
  using L = Lam<PREC>;
  using ::fma;
  const int n = blockIdx.x * kBlock + threadIdx.x;
  if (n >= N) return;
  int m[18];
  if (RIA) {
    nbr_ria(t, ria_locate(t, n), m);
  } else {
    nbr_adj(t, n, m);
  }
  // forward quantities of F_n
  R d[kQ];
  gather<PREC, false>(G, t.npad, n, m, d, kp.inv_scale, cc, t.pressure);
  R drho = d[0], jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    drho += d[i];
    if (cx(i)) jx += cx(i) > 0 ? d[i] : -d[i];
    if (cy(i)) jy += cy(i) > 0 ? d[i] : -d[i];
    if (cz(i)) jz += cz(i) > 0 ? d[i] : -d[i];
  }
  const R rho = c.rho_s + drho;
  const R irho = recip(rho);
  const R sn = DRAG ? R(__ldg(s + n)) : R(0);
  const R kd = DRAG ? recip(R(1) + half(sn)) : R(1);
  const R ux = fma(jx, irho, c.hg[0]) * kd, uy = fma(jy, irho, c.hg[1]) * kd, uz = fma(jz, irho, c.hg[2]) * kd;
  // mu = S^T lambda_{n+1}: slot (j, n) of the post-collision state is pulled by
  // node m_{inv j} (fluid) or, through a marker, by this node's inv j slot
  // (sign -1 for anti-bounce-back).
  R mu[kQ];
  mu[0] = L::ld(lam_next + n);
#pragma unroll
  for (int j = 1; j < kQ; ++j) {
    const int mp = m[inv(j) - 1];
    const int dir = mp >= 0 ? j : inv(j);
    const int node = mp >= 0 ? mp : n;
    const R v = L::ld(lam_next + at(dir, t.npad, node));
    mu[j] = mp < -1 ? -v : v;
  }
  // weighted moments of mu (pairs: even part for M0/M2, odd part for M1)
  R M0 = c.w[0] * mu[0];
  R M1x = R(0), M1y = R(0), M1z = R(0);
  R Mxx = R(0), Myy = R(0), Mzz = R(0), Mxy = R(0), Mxz = R(0), Myz = R(0);
#pragma unroll
  for (int k = 1; k <= 9; ++k) {
    const int a = 2 * k - 1;
    const R w = c.w[wclass(a)];
    const R sp = w * (mu[a] + mu[a + 1]);
    const R sm = w * (mu[a] - mu[a + 1]);
    M0 += sp;
    if (cx(a)) M1x += cx(a) > 0 ? sm : -sm;
    if (cy(a)) M1y += cy(a) > 0 ? sm : -sm;
    if (cz(a)) M1z += cz(a) > 0 ? sm : -sm;
    if (cx(a)) Mxx += sp;
    if (cy(a)) Myy += sp;
    if (cz(a)) Mzz += sp;
    if (cx(a) && cy(a)) Mxy += cx(a) * cy(a) > 0 ? sp : -sp;
    if (cx(a) && cz(a)) Mxz += cx(a) * cz(a) > 0 ? sp : -sp;
    if (cy(a) && cz(a)) Myz += cy(a) * cz(a) > 0 ? sp : -sp;
  }
  const R M2ux = fma(Mxx, ux, fma(Mxy, uy, Mxz * uz));
  const R M2uy = fma(Mxy, ux, fma(Myy, uy, Myz * uz));
  const R M2uz = fma(Mxz, ux, fma(Myz, uy, Mzz * uz));
  const R M2gx = fma(Mxx, c.g[0], fma(Mxy, c.g[1], Mxz * c.g[2]));
  const R M2gy = fma(Mxy, c.g[0], fma(Myy, c.g[1], Myz * c.g[2]));
  const R M2gz = fma(Mxz, c.g[0], fma(Myz, c.g[1], Mzz * c.g[2]));
  const R uu = fma(ux, ux, fma(uy, uy, uz * uz));
  const R q = fma(ux, M2ux, fma(uy, M2uy, uz * M2uz));
  const R av = fma(M1x, ux, fma(M1y, uy, M1z * uz));
  const R ug = fma(ux, c.g[0], fma(uy, c.g[1], uz * c.g[2]));
  const R uM2g = fma(ux, M2gx, fma(uy, M2gy, uz * M2gz));
  const R M1g = fma(M1x, c.g[0], fma(M1y, c.g[1], M1z * c.g[2]));
  const R lp = c.lp, lm = c.lm, ap = c.ap, am = c.am;
  const R lpM0 = lp * M0, apM0 = ap * M0;
  // Psi and dPsi/du (see the header comment)
  R Psi = lpM0 * fma(-1.5f * uu, R(1), R(1)) + 4.5f * (lp * q) + 3.0f * (lm * av) + 9.0f * (ap * uM2g) -
          3.0f * (apM0 * ug) + 3.0f * (am * M1g);
  R Px = -3.0f * (lpM0 * ux) + 9.0f * (lp * M2ux) + 3.0f * (lm * M1x) + 9.0f * (ap * M2gx) - 3.0f * (apM0 * c.g[0]);
  R Py = -3.0f * (lpM0 * uy) + 9.0f * (lp * M2uy) + 3.0f * (lm * M1y) + 9.0f * (ap * M2gy) - 3.0f * (apM0 * c.g[1]);
  R Pz = -3.0f * (lpM0 * uz) + 9.0f * (lp * M2uz) + 3.0f * (lm * M1z) + 9.0f * (ap * M2gz) - 3.0f * (apM0 * c.g[2]);
  const R dPsi_ds = -9.0f * (ap * q) + 3.0f * (apM0 * uu) - 3.0f * (am * av);
  if (DRAG) {
    Psi += sn * dPsi_ds;
    Px += sn * (-18.0f * (ap * M2ux) + 6.0f * (apM0 * ux) - 3.0f * (am * M1x));
    Py += sn * (-18.0f * (ap * M2uy) + 6.0f * (apM0 * uy) - 3.0f * (am * M1y));
    Pz += sn * (-18.0f * (ap * M2uz) + 6.0f * (apM0 * uz) - 3.0f * (am * M1z));
  }
  const R A = Psi - (Px * (ux - kd * c.hg[0]) + Py * (uy - kd * c.hg[1]) + Pz * (uz - kd * c.hg[2]));
  const R Bx = kd * Px, By = kd * Py, Bz = kd * Pz;
  if (grad_s) {
    const R gs = rho * (dPsi_ds - half(kd) * (Px * ux + Py * uy + Pz * uz));
    grad_s[n] += L::to_double(gs);
  }
  L::st(lam + n, fma(c.omlp, mu[0], A));
#pragma unroll
  for (int k = 1; k <= 9; ++k) {
    const int a = 2 * k - 1;
    const R sp = mu[a] + mu[a + 1], sm = mu[a] - mu[a + 1];
    R Bc = R(0);
    if (cx(a)) Bc += cx(a) > 0 ? Bx : -Bx;
    if (cy(a)) Bc += cy(a) > 0 ? By : -By;
    if (cz(a)) Bc += cz(a) > 0 ? Bz : -Bz;
    const R e = fma(c.qp, sp, A);
    const R o = fma(c.qm, sm, Bc);
    L::st(lam + at(a, t.npad, n), e + o);
    L::st(lam + at(a + 1, t.npad, n), e - o);
  }
}

// Compensated (two-sum) block reduction of one double; result in thread 0.
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void block_sum_dd(double& hi, double& lo, double (*s_red)[2]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double h2 = __shfl_down_sync(0xffffffffu, hi, o), l2 = __shfl_down_sync(0xffffffffu, lo, o);
    double s, e;
    two_sum(hi, h2, s, e);
    hi = s;
    lo = lo + l2 + e;
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    s_red[w][0] = hi;
    s_red[w][1] = lo;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double H = s_red[0][0], Lo = s_red[0][1];
    for (int j = 1; j < int(blockDim.x >> 5); ++j) {
      double s, e;
      two_sum(H, s_red[j][0], s, e);
      H = s;
      Lo += s_red[j][1] + e;
    }
    hi = H;
    lo = Lo;
  }
}

// J partial sums of rho u_x (compensated), optional dJ/dF_T and the direct dJ/ds.
template <int PREC, bool RIA>
__global__ void __launch_bounds__(kBlock) k_objective(DevTables t, KParams kp, CollConst<typename St<PREC>::R> c,
                                                      const typename St<PREC>::T* pdf, int layout,
                                                      const float* __restrict__ s, double invN,
                                                      double* __restrict__ partials,
                                                      typename St<PREC>::R* __restrict__ lamT,
                                                      double* __restrict__ grad_s, int N) {
  using R = typename St<PREC>::R;
  __shared__ double s_red[kBlock / 32][2];
  const int n0 = blockIdx.x * kBlock;
  const int n = n0 + threadIdx.x;
  double f[kQ];
  double hi = 0.0, lo = 0.0;
  if (node_canonical<PREC, RIA>(t, kp, c, pdf, layout, n, N, f)) {
    double r = 0.0, jx = 0.0;
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      r += f[i];
      if (cx(i)) jx += cx(i) > 0 ? f[i] : -f[i];
    }
    const double kd = s ? 1.0 / (1.0 + 0.5 * double(s[n])) : 1.0;
    const double rux = (jx + 0.5 * kp.g[0] * r) * kd;  // rho u_x
    hi = rux;
    if (lamT) {
#pragma unroll
      for (int i = 0; i < kQ; ++i) lamT[at(i, t.npad, n)] = R((cx(i) + 0.5 * kp.g[0]) * kd * invN);
    }
    if (grad_s) grad_s[n] = -0.5 * rux * kd * invN;
  }
  __syncthreads();
  block_sum_dd(hi, lo, s_red);
  if (threadIdx.x == 0) {
    partials[2 * size_t(blockIdx.x)] = hi;
    partials[2 * size_t(blockIdx.x) + 1] = lo;
  }
}

template <int PREC>
__global__ void __launch_bounds__(512) k_finish_dd(const double* __restrict__ partials, int64_t nparts, double scale,
                                                   double* __restrict__ out) {
  __shared__ double s_red[16][2];
  double hi = 0.0, lo = 0.0;
  for (int64_t p = threadIdx.x; p < nparts; p += blockDim.x) {
    double s, e;
    two_sum(hi, partials[2 * p], s, e);
    hi = s;
    lo += partials[2 * p + 1] + e;
  }
  block_sum_dd(hi, lo, s_red);
  if (threadIdx.x == 0) out[0] = (hi + lo) * scale;
}

}  // namespace dev

template <int PREC>
int launch_adjoint_t(const lbm_lattice* L, const KParams& kp, const void* G, const void* lam_next, void* lam,
                     const float* s, double* grad_s, int ria, void* stream) {
  using T = typename dev::St<PREC>::T;
  using R = typename dev::St<PREC>::R;
  using LT = typename dev::Lam<PREC>::T;
  auto st = static_cast<cudaStream_t>(stream);
  const auto cc = dev::make_coll<R>(kp);
  const auto ac = dev::make_adj<R>(kp);
  const unsigned g = grid_of(L->N);
  const T* Gp = static_cast<const T*>(G);
  const LT* ln = static_cast<const LT*>(lam_next);
  LT* lo = static_cast<LT*>(lam);
  const int N = int(L->N);
#define LBM_ADJ(R_, D_) dev::k_adjoint<PREC, R_, D_><<<g, dev::kBlock, 0, st>>>(L->dev, kp, cc, ac, Gp, ln, lo, s, grad_s, N)
  if (s) {
    if (ria) LBM_ADJ(true, true); else LBM_ADJ(false, true);
  } else {
    if (ria) LBM_ADJ(true, false); else LBM_ADJ(false, false);
  }
#undef LBM_ADJ
  return cuda_check("adjoint step launch");
}

template <int PREC>
int launch_objective_t(const lbm_lattice* L, const KParams& kp, const void* pdf, int layout, const float* s,
                       double* J, void* lamT, double* grad_s, double* partials, void* stream) {
  using T = typename dev::St<PREC>::T;
  using R = typename dev::St<PREC>::R;
  auto st = static_cast<cudaStream_t>(stream);
  const int64_t parts = reduce_parts(L);
  const double invN = L->N > 0 ? 1.0 / double(L->N) : 0.0;
  if (L->N > 0) {
    const bool ria = !(L->uploaded & LBM_TABLES_ADJ);
    const auto c = dev::make_coll<R>(kp);
    if (ria)
      dev::k_objective<PREC, true><<<grid_of(L->N), dev::kBlock, 0, st>>>(
          L->dev, kp, c, static_cast<const T*>(pdf), layout, s, invN, partials, static_cast<R*>(lamT), grad_s,
          int(L->N));
    else
      dev::k_objective<PREC, false><<<grid_of(L->N), dev::kBlock, 0, st>>>(
          L->dev, kp, c, static_cast<const T*>(pdf), layout, s, invN, partials, static_cast<R*>(lamT), grad_s,
          int(L->N));
    if (int rc = cuda_check("objective launch")) return rc;
  }
  dev::k_finish_dd<PREC><<<1, 512, 0, st>>>(partials, L->N > 0 ? parts : 0, invN, J);
  return cuda_check("objective reduction launch");
}

template int launch_adjoint_t<LBM_F64>(const lbm_lattice*, const KParams&, const void*, const void*, void*,
                                       const float*, double*, int, void*);
template int launch_adjoint_t<LBM_F32>(const lbm_lattice*, const KParams&, const void*, const void*, void*,
                                       const float*, double*, int, void*);
template int launch_adjoint_t<LBM_F16S>(const lbm_lattice*, const KParams&, const void*, const void*, void*,
                                        const float*, double*, int, void*);
template int launch_adjoint_t<LBM_F64_DF>(const lbm_lattice*, const KParams&, const void*, const void*, void*,
                                          const float*, double*, int, void*);
template int launch_objective_t<LBM_F64>(const lbm_lattice*, const KParams&, const void*, int, const float*, double*,
                                         void*, double*, double*, void*);
template int launch_objective_t<LBM_F32>(const lbm_lattice*, const KParams&, const void*, int, const float*, double*,
                                         void*, double*, double*, void*);
template int launch_objective_t<LBM_F16S>(const lbm_lattice*, const KParams&, const void*, int, const float*,
                                          double*, void*, double*, double*, void*);

}  // namespace lbm
