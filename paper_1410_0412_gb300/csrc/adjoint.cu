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
  // integer multiples of the rates, folded once on the host
  R k45lp, k9lp, nk3lp;     // 9/2 l+, 9 l+, -3 l+
  R k3lm;                   // 3 l-
  R k9ap, nk3ap, nk9ap;     // 9 a+, -3 a+, -9 a+
  R nk18ap, k6ap;           // -18 a+, 6 a+
  R k3am, nk3am;            // 3 a-, -3 a-
  bool gx;                  // the body force points along x (g_y = g_z = 0)
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
  const double ap = 1.0 - kp.lp / 2, am = 1.0 - kp.lm / 2;
  c.k45lp = R(4.5 * kp.lp);
  c.k9lp = R(9.0 * kp.lp);
  c.nk3lp = R(-3.0 * kp.lp);
  c.k3lm = R(3.0 * kp.lm);
  c.k9ap = R(9.0 * ap);
  c.nk3ap = R(-3.0 * ap);
  c.nk9ap = R(-9.0 * ap);
  c.nk18ap = R(-18.0 * ap);
  c.k6ap = R(6.0 * ap);
  c.k3am = R(3.0 * am);
  c.nk3am = R(-3.0 * am);
  c.gx = kp.g[1] == 0.0 && kp.g[2] == 0.0;
  return c;
}

// Pair sums P_k = mu_a + mu_b and differences D_k = mu_a - mu_b of the adjoint
// vector and its weighted moments M0 = sum w mu, M1 = sum w c mu and
// M2 = sum w c c^T mu.  The diagonal weight w2 = 1/36 is half the axis weight,
// so each moment is w2 times an integer-coefficient sum of P_k or D_k (plus
// w0 mu_0 for M0).  FP64 forms those sums exactly in fixed point on the
// integer pipe (exact64.cuh) and rounds each once; P_k is converted only when
// the caller needs it (l+ != 1).
// NEED_PD: convert P and D to R (the FP64 pair update needs them; the
// fixed-point one reads the integers Pi, Di at the scale emax instead).
template <class R, bool NEED_P, bool NEED_PD = true>
__device__ __forceinline__ void adj_moments(const R (&mu)[kQ], const AdjConst<R>& c, R (&P)[10], R (&D)[10], R& M0,
                                            R& M1x, R& M1y, R& M1z, R& Mxx, R& Myy, R& Mzz, R& Mxy, R& Mxz,
                                            R& Myz, int64_t (&Pi)[10], int64_t (&Di)[10], int& emax) {
  using ::fma;
  const R w2 = c.w[2];
  if constexpr (std::is_same<R, double>::value) {
    uint64_t b[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) b[i] = dbits(mu[i]);
    emax = fx_scale(b);
    int64_t f[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) f[i] = fx_of(b[i], emax);
#pragma unroll
    for (int k = 1; k <= 9; ++k) {
      Pi[k] = f[2 * k - 1] + f[2 * k];
      Di[k] = f[2 * k - 1] - f[2 * k];
      if (NEED_PD && NEED_P) P[k] = fx_to_double(Pi[k], emax);
      if (NEED_PD) D[k] = fx_to_double(Di[k], emax);
    }
    // every integer sum below has at most 24 terms of magnitude < 2^58
    const int64_t A1 = Pi[1] + Pi[2] + Pi[3];
    const int64_t A2 = Pi[4] + Pi[5] + Pi[6] + Pi[7] + Pi[8] + Pi[9];
    M0 = fma(c.w[0], mu[0], w2 * fx_to_double(2 * A1 + A2, emax));
    if (emax >= kFxMaxExp) M0 = dfrom(0x7ff8000000000000ull);
    M1x = w2 * fx_to_double(2 * Di[1] + Di[4] + Di[5] + Di[6] + Di[7], emax);
    M1y = w2 * fx_to_double(2 * Di[2] + Di[4] - Di[5] + Di[8] + Di[9], emax);
    M1z = w2 * fx_to_double(2 * Di[3] + Di[6] - Di[7] + Di[8] - Di[9], emax);
    Mxx = w2 * fx_to_double(2 * Pi[1] + Pi[4] + Pi[5] + Pi[6] + Pi[7], emax);
    Myy = w2 * fx_to_double(2 * Pi[2] + Pi[4] + Pi[5] + Pi[8] + Pi[9], emax);
    Mzz = w2 * fx_to_double(2 * Pi[3] + Pi[6] + Pi[7] + Pi[8] + Pi[9], emax);
    Mxy = w2 * fx_to_double(Pi[4] - Pi[5], emax);
    Mxz = w2 * fx_to_double(Pi[6] - Pi[7], emax);
    Myz = w2 * fx_to_double(Pi[8] - Pi[9], emax);
  } else {
#pragma unroll
    for (int k = 1; k <= 9; ++k) {
      P[k] = mu[2 * k - 1] + mu[2 * k];
      D[k] = mu[2 * k - 1] - mu[2 * k];
    }
    const R A1 = P[1] + P[2] + P[3];
    const R A2 = (P[4] + P[5]) + (P[6] + P[7]) + (P[8] + P[9]);
    M0 = fma(c.w[0], mu[0], w2 * (A1 + A1 + A2));
    M1x = w2 * ((D[1] + D[1]) + ((D[4] + D[5]) + (D[6] + D[7])));
    M1y = w2 * ((D[2] + D[2]) + ((D[4] - D[5]) + (D[8] + D[9])));
    M1z = w2 * ((D[3] + D[3]) + ((D[6] - D[7]) + (D[8] - D[9])));
    Mxx = w2 * ((P[1] + P[1]) + ((P[4] + P[5]) + (P[6] + P[7])));
    Myy = w2 * ((P[2] + P[2]) + ((P[4] + P[5]) + (P[8] + P[9])));
    Mzz = w2 * ((P[3] + P[3]) + ((P[6] + P[7]) + (P[8] + P[9])));
    Mxy = w2 * (P[4] - P[5]);
    Mxz = w2 * (P[6] - P[7]);
    Myz = w2 * (P[8] - P[9]);
  }
}

// One adjoint step.  G: OS-NT grid at step n (its pull gather is F_n).
// lam_next / lam: adjoint of the canonical states F_{n+1} / F_n, layout [19][Npad].
// LP1: l+ = 1 (FP64-storage paths), where (1 - l+)/2 = 1 - l+ = 0.
template <int PREC, bool RIA, bool DRAG, bool LP1 = false>
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
  // F_n (the OS-NT pull gather of G) and mu = S^T lambda_{n+1}: slot (j, n) of
  // the post-collision state is pulled by node m_{inv j} (fluid) or, through a
  // marker, by this node's inv j slot (sign -1 for anti-bounce-back).
  R d[kQ], mu[kQ];
  if (RIA && t.run_slot) {
    // Run slots (no pressure faces, the grid below 2^31 slots): the pull slots
    // of F_n are run_slot_osnt(i, r) + off, and the slot of lambda_{n+1} that
    // direction j reads is the AA odd table's run_slot(inv j, r) + off.
    const RiaCursor cur = ria_locate<kKeepIdx<PREC>>(t, n);
    unsigned sl[18];
    run_slots<kKeepIdx<PREC>>(t.run_slot_osnt, t.rpad, cur.r, cur.off, sl);
    d[0] = St<PREC>::ld(G + n, kp.inv_scale);
#pragma unroll
    for (int i = 1; i < kQ; ++i) d[i] = St<PREC>::ld(G + sl[i - 1], kp.inv_scale);
    run_slots<kKeepIdx<PREC>>(t.run_slot, t.rpad, cur.r, cur.off, sl);
    mu[0] = L::ld(lam_next + n);
#pragma unroll
    for (int j = 1; j < kQ; ++j) mu[j] = L::ld(lam_next + sl[inv(j) - 1]);
  } else {
    int m[18];
    if (RIA) {
      nbr_ria(t, ria_locate(t, n), m);
    } else {
      nbr_adj(t, n, m);
    }
    gather<PREC, false>(G, t.npad, n, m, d, kp.inv_scale, cc.abb_in, cc.abb_out, t.pressure);
    mu[0] = L::ld(lam_next + n);
#pragma unroll
    for (int j = 1; j < kQ; ++j) {
      const int mp = m[inv(j) - 1];
      const int dir = mp >= 0 ? j : inv(j);
      const int node = mp >= 0 ? mp : n;
      const R v = L::ld(lam_next + at(dir, t.npad, node));
      mu[j] = mp < -1 ? -v : v;
    }
  }
  R sa[10], da[10], drho, jx, jy, jz;
  moments<R, false>(d, sa, da, drho, jx, jy, jz);
  const R rho = c.rho_s + drho;
  const R irho = recip(rho);
  const R sn = DRAG ? R(__ldg(s + n)) : R(0);
  const R kd = DRAG ? recip(R(1) + halve(sn)) : R(1);
  R ux = fma(jx, irho, c.hg[0]), uy = fma(jy, irho, c.hg[1]), uz = fma(jz, irho, c.hg[2]);
  if (DRAG) {
    ux *= kd;
    uy *= kd;
    uz *= kd;
  }
  R P[10], D[10], M0, M1x, M1y, M1z, Mxx, Myy, Mzz, Mxy, Mxz, Myz;
  int64_t Pi[10], Di[10];
  int emax_mu = 0;
  constexpr bool kFxOut = std::is_same<R, double>::value;  // the fixed-point pair update below
  adj_moments<R, !LP1, !kFxOut>(mu, c, P, D, M0, M1x, M1y, M1z, Mxx, Myy, Mzz, Mxy, Mxz, Myz, Pi, Di, emax_mu);
  const R M2ux = fma(Mxx, ux, fma(Mxy, uy, Mxz * uz));
  const R M2uy = fma(Mxy, ux, fma(Myy, uy, Myz * uz));
  const R M2uz = fma(Mxz, ux, fma(Myz, uy, Mzz * uz));
  const R uu = fma(ux, ux, fma(uy, uy, uz * uz));
  const R q = fma(ux, M2ux, fma(uy, M2uy, uz * M2uz));
  const R av = fma(M1x, ux, fma(M1y, uy, M1z * uz));
  const R apM0 = c.ap * M0;
  const R nk3lpM0 = c.nk3lp * M0, nk3apM0 = c.nk3ap * M0;  // -3 l+ M0, -3 a+ M0
  // the force terms: M2 g, u.g, u.M2 g, M1.g and -3 a+ M0 g
  R M2gx, M2gy, M2gz, ug, M1g, Gx, Gy, Gz;
  if (std::is_same<R, double>::value && c.gx) {  // uniform: a force along x alone
    M2gx = Mxx * c.g[0];
    M2gy = Mxy * c.g[0];
    M2gz = Mxz * c.g[0];
    ug = ux * c.g[0];
    M1g = M1x * c.g[0];
    Gx = nk3apM0 * c.g[0];
    Gy = R(0);
    Gz = R(0);
  } else {
    M2gx = fma(Mxx, c.g[0], fma(Mxy, c.g[1], Mxz * c.g[2]));
    M2gy = fma(Mxy, c.g[0], fma(Myy, c.g[1], Myz * c.g[2]));
    M2gz = fma(Mxz, c.g[0], fma(Myz, c.g[1], Mzz * c.g[2]));
    ug = fma(ux, c.g[0], fma(uy, c.g[1], uz * c.g[2]));
    M1g = fma(M1x, c.g[0], fma(M1y, c.g[1], M1z * c.g[2]));
    Gx = nk3apM0 * c.g[0];
    Gy = nk3apM0 * c.g[1];
    Gz = nk3apM0 * c.g[2];
  }
  const R uM2g = fma(ux, M2gx, fma(uy, M2gy, uz * M2gz));
  // Psi and dPsi/du (see the header comment)
  R Psi = fma(c.lp * M0, fma(R(-1.5f), uu, R(1)),
              fma(c.k45lp, q, fma(c.k3lm, av, fma(c.k9ap, uM2g, fma(c.k3am, M1g, nk3apM0 * ug)))));
  R Px = fma(nk3lpM0, ux, fma(c.k9lp, M2ux, fma(c.k3lm, M1x, fma(c.k9ap, M2gx, Gx))));
  R Py = fma(nk3lpM0, uy, fma(c.k9lp, M2uy, fma(c.k3lm, M1y, fma(c.k9ap, M2gy, Gy))));
  R Pz = fma(nk3lpM0, uz, fma(c.k9lp, M2uz, fma(c.k3lm, M1z, fma(c.k9ap, M2gz, Gz))));
  const R dPsi_ds = fma(c.nk9ap, q, fma(R(3), apM0 * uu, c.nk3am * av));
  if (DRAG) {
    Psi = fma(sn, dPsi_ds, Psi);
    const R k6apM0 = c.k6ap * M0;
    Px = fma(sn, fma(c.nk18ap, M2ux, fma(k6apM0, ux, c.nk3am * M1x)), Px);
    Py = fma(sn, fma(c.nk18ap, M2uy, fma(k6apM0, uy, c.nk3am * M1y)), Py);
    Pz = fma(sn, fma(c.nk18ap, M2uz, fma(k6apM0, uz, c.nk3am * M1z)), Pz);
  }
  // A = Psi - P.(u - kd g/2)
  const R A = fma(-Px, fma(-kd, c.hg[0], ux), fma(-Py, fma(-kd, c.hg[1], uy), fma(-Pz, fma(-kd, c.hg[2], uz), Psi)));
  const R Bx = kd * Px, By = kd * Py, Bz = kd * Pz;
  if (grad_s) {
    const R Pu = fma(Px, ux, fma(Py, uy, Pz * uz));
    const R gs = rho * fma(-halve(kd), Pu, dPsi_ds);
    grad_s[n] += L::to_double(gs);
  }
  L::st(lam + n, LP1 ? A : fma(c.omlp, mu[0], A));
  if constexpr (kFxOut) {
    // The pair update lambda_a,b = e +- o, e = A + qp P_k, o = qm D_k + c_a.B, in
    // 64-bit fixed point at one bit finer than the adjoint moments' scale:
    // P_k and D_k enter exactly, A and B truncated, the products floored,
    // each output rounded once.  |mu_i| < 2 B_mu gives |D_k|, |P_k| < 4 B_mu;
    // with |A|, |B_a| < 4 B_mu (checked) every value stays below 16 B_mu, half
    // the int64 range at this scale.  Otherwise the warp takes the FP64 update.
    constexpr int kxa = 1;
    const bool ok = emax_mu < kFxMaxExp && dexp(A) <= emax_mu + 1 && dexp(Bx) <= emax_mu + 1 &&
                    dexp(By) <= emax_mu + 1 && dexp(Bz) <= emax_mu + 1;
    if (__all_sync(__activemask(), ok)) {
      const int es = emax_mu - kxa;
      const int64_t Af = fx_of(dbits(A), es);
      const int64_t Bxf = fx_of(dbits(Bx), es), Byf = fx_of(dbits(By), es), Bzf = fx_of(dbits(Bz), es);
#pragma unroll
      for (int k = 1; k <= 9; ++k) {
        const int a = 2 * k - 1;
        const int64_t Bc = k == 1 ? Bxf : k == 2 ? Byf : k == 3 ? Bzf : k == 4 ? Bxf + Byf : k == 5 ? Bxf - Byf
                         : k == 6 ? Bxf + Bzf : k == 7 ? Bxf - Bzf : k == 8 ? Byf + Bzf : Byf - Bzf;
        const int64_t Df = static_cast<int64_t>(static_cast<uint64_t>(Di[k]) << kxa);
        int64_t e = Af;
        if (!LP1) e += mulhi_q64(cc.qp_fx, static_cast<int64_t>(static_cast<uint64_t>(Pi[k]) << kxa));
        const int64_t o = mulhi_q64(cc.qm_fx, Df) + Bc;
        L::st(lam + at(a, t.npad, n), fx_to_double(e + o, es));
        L::st(lam + at(a + 1, t.npad, n), fx_to_double(e - o, es));
      }
      return;
    }
#pragma unroll
    for (int k = 1; k <= 9; ++k) {
      if (!LP1) P[k] = fx_to_double(Pi[k], emax_mu);
      D[k] = fx_to_double(Di[k], emax_mu);
    }
  }
#pragma unroll
  for (int k = 1; k <= 9; ++k) {
    const int a = 2 * k - 1;
    // c_a . B for the pair's first direction (the loop is unrolled: k is a constant)
    const R Bc = k == 1 ? Bx : k == 2 ? By : k == 3 ? Bz : k == 4 ? Bx + By : k == 5 ? Bx - By
               : k == 6 ? Bx + Bz : k == 7 ? Bx - Bz : k == 8 ? By + Bz : By - Bz;
    const R e = LP1 ? A : fma(c.qp, P[k], A);
    const R o = fma(c.qm, D[k], Bc);
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
  if (node_canonical<PREC, RIA, false>(t, kp, c, pdf, layout, n, N, f)) {
    // rho and j_x from the stored values as exact fixed-point sums, each
    // rounded once (exact64.cuh): the objective's per-node terms carry no
    // summation error, which keeps finite differences of J above round-off
    int64_t Sk[10], D[10], S, Jx, Jy, Jz;
    const int emax = fx_moments<false>(f, Sk, D, S, Jx, Jy, Jz);
    const double r = kp.rho_s + (emax < kFxMaxExp ? fx_to_double(S, emax) : dfrom(0x7ff8000000000000ull));
    const double jx = fx_to_double(Jx, emax);
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
  const unsigned blk = dev::kBlock;
  const unsigned g = grid_of(L->N);
  const T* Gp = static_cast<const T*>(G);
  const LT* ln = static_cast<const LT*>(lam_next);
  LT* lo = static_cast<LT*>(lam);
  const int N = int(L->N);
  const bool lp1 = use_lp1<PREC>(kp);
#define LBM_ADJ(R_, D_) LBM_LAUNCH_LP1(k_adjoint, LBM_TARGS2(R_, D_), (L->dev, kp, cc, ac, Gp, ln, lo, s, grad_s, N))
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
