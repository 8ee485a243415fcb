// smc_models.cuh -- the built-in PCFG block tables (the B, S and sim of
// Section 3.1) and the per-warp PC-sorted dispatch loop that runs them.
//
// A model supplies:
//   Lane           per-particle registers for one segment (PSTATE fields that
//                  cross checkpoints plus segment-local scratch);
//   init/gather/store  PSTATE <-> registers (gather = Section 3.3's particle
//                  duplication, reading the ancestor's slot of the SoA arrays);
//   block(b, ...)  one basic block; sets pc to the successor and `ckpt` when
//                  the block ends in a checkpoint (Algorithm 1's c_n).
// Block index PC_STOP (-1) is b_stop: sim(b_stop, s) = (b_stop, s, true).
#pragma once
#include "../../include/smc.h"
#include "smc_device.cuh"

namespace smc {

// Model constants resident in device memory (Section 3.3: observations and
// the tree are shared global constants, not per-particle state).
// The observed branch of segment k of a tree model, precomputed on the host in
// traversal order so that a branch block makes one 32-byte load instead of a
// chain of dependent ones: node v = preorder[k], its parent's age (start) and
// its own (stop), bit 0 of flags: v is internal, bit 1: v is its parent's left
// child.
struct BranchRec {
  double start, stop;
  int v, flags;
  long long pad_;
};

__device__ __forceinline__ BranchRec load_branch(const BranchRec* __restrict__ b, int k) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(b + k));
  const int4 c = __ldg(reinterpret_cast<const int4*>(b + k) + 1);
  return BranchRec{a.x, a.y, c.x, c.y, 0};
}

struct ModelDev {
  int kind, T, n_nodes, fixed_rates, depth_cap, call_limit, lam_stack_cap, pad_;
  const MathTab* tab;  // this device's log / exp tables
  double log_rho;      // log(rho), computed on the host
  const double* obs;
  const BranchRec* branch;  // tree models: [n_nodes], entry k for k >= 1
  const int* parent;
  const int* left;
  const int* preorder;
  const double* age;
  const double* fixed_mult;
  double x0_mean, x0_sd, a, b, q_sd, r_sd, lg_lc, corr;
  double rho, lambda_fixed, mu_fixed, lambda_scale, mu_scale, sigma, geo_p, geo_logw;
};

// One buffer of the double-buffered SoA PSTATE (Section 3.3's separate arrays
// per field): real fields [n_real][N], int fields [n_int][N] (field 0 = block
// index), stack rows [cap][N].  Field-major with particle index fastest so a
// warp touches 32 consecutive elements of every field.
struct StateView {
  void* real;
  int32_t* ints;
  void* stack;
  template <typename R>
  __device__ __forceinline__ R& rf(int f, int i, int N) const {
    return reinterpret_cast<R*>(real)[(size_t)f * N + i];
  }
  __device__ __forceinline__ int32_t& inf_(int f, int i, int N) const {
    return ints[(size_t)f * N + i];
  }
  template <typename R>
  __device__ __forceinline__ R& st(int s, int i, int N) const {
    return reinterpret_cast<R*>(stack)[(size_t)s * N + i];
  }
};

// A snapshot of a population in smc_result's output layouts (device memory):
// log-weights [N], real fields [n_real][N] (f64), int fields [n_int][N], stack
// rows [cap][N] (f64).  A model's load() puts particle i of it into the lane and
// into the state buffer being written (its stack rows).
struct SnapView {
  const double* logw;
  const double* real;
  const int32_t* ints;
  const double* stack;
};

// ------------------------------------------------------------------------
// Linear-Gaussian state-space model (Eq. 2 family, blocks of Fig. 3):
//   block 0 `init`: x = x0_mean + x0_sd z, then a non-checkpoint jump to iter;
//   block 1 `iter`: x = a x + (b + q_sd z); observe y_k ~ N(x, r_sd^2);
//                   checkpoint; NEXT = b_stop after the T-th observation.
// The observation index equals the checkpoint index k (all particles reach
// every checkpoint together), so t is not stored per particle.
// ------------------------------------------------------------------------
template <typename Real>
struct LgModel {
  using R = Real;
  static constexpr int NB = 2, N_REAL = 1, N_INT = 1;
  static constexpr bool HAS_STACK = false;
  struct Lane {
    int pc;
    bool ckpt;
    R x, logw;
    int overflow, limited;
  };
  __device__ static void init(Lane& L) {
    L.pc = 0;
    L.x = (R)0;
    L.logw = (R)0;
  }
  __device__ static void gather(Lane& L, const StateView& Sc, const StateView&, int a, int, int N,
                                const ModelDev&) {
    L.x = Sc.rf<R>(0, a, N);
    L.pc = Sc.inf_(0, a, N);
    L.logw = (R)0;
  }
  __device__ static void store(const Lane& L, const StateView& Sn, int i, int N) {
    Sn.rf<R>(0, i, N) = L.x;
    Sn.inf_(0, i, N) = L.pc;
  }
  __device__ static void load(Lane& L, const StateView&, const SnapView& P, int i, int N,
                              const Stream&) {
    L.x = (R)P.real[i];
    L.pc = P.ints[i];
    L.logw = (R)P.logw[i];
  }
  __device__ static void begin(Lane& L) {
    L.ckpt = false;
    L.overflow = L.limited = 0;
  }
  __device__ static void block(int b, Lane& L, Stream& s, const ModelDev& md, const StateView&, int,
                               int k, int) {
    if (b == 0) {
      const R z0 = normal01<R>(s);
      L.x = m_fma((R)md.x0_sd, z0, (R)md.x0_mean);
      L.pc = 1;
      return;
    }
    const R z = normal01<R>(s);
    L.x = m_fma((R)md.a, L.x, m_fma((R)md.q_sd, z, (R)md.b));
    const R y = (R)md.obs[k];
    const R dz = (y - L.x) / (R)md.r_sd;
    const R lp = (R)-0.5 * (dz * dz) - (R)md.lg_lc;
    L.logw = L.logw + lp;
    L.pc = (k + 1 == md.T) ? PC_STOP : 1;
    L.ckpt = true;
  }
};

// ------------------------------------------------------------------------
// Weighted geometric program (Fig. 2a) with a checkpoint after every flip:
// block 0 flips Bernoulli(p); heads -> weight geo_logw and loop, tails ->
// b_stop.  Particles finish at different checkpoints; finished ones keep
// taking part in resampling.
// ------------------------------------------------------------------------
template <typename Real>
struct GeoModel {
  using R = Real;
  static constexpr int NB = 1, N_REAL = 0, N_INT = 2;
  static constexpr bool HAS_STACK = false;
  struct Lane {
    int pc, count;
    bool ckpt;
    R logw;
    int overflow, limited;
  };
  __device__ static void init(Lane& L) {
    L.pc = 0;
    L.count = 0;
    L.logw = (R)0;
  }
  __device__ static void gather(Lane& L, const StateView& Sc, const StateView&, int a, int, int N,
                                const ModelDev&) {
    L.pc = Sc.inf_(0, a, N);
    L.count = Sc.inf_(1, a, N);
    L.logw = (R)0;
  }
  __device__ static void store(const Lane& L, const StateView& Sn, int i, int N) {
    Sn.inf_(0, i, N) = L.pc;
    Sn.inf_(1, i, N) = L.count;
  }
  __device__ static void load(Lane& L, const StateView&, const SnapView& P, int i, int N,
                              const Stream&) {
    L.pc = P.ints[i];
    L.count = P.ints[(size_t)N + i];
    L.logw = (R)P.logw[i];
  }
  __device__ static void begin(Lane& L) {
    L.ckpt = false;
    L.overflow = L.limited = 0;
  }
  __device__ static void block(int, Lane& L, Stream& s, const ModelDev& md, const StateView&, int,
                               int, int) {
    const bool heads = bernoulli<R>(s, (R)md.geo_p);
    L.count += 1;
    if (heads) {
      L.logw = L.logw + (R)md.geo_logw;
      L.pc = 0;
    } else {
      L.pc = PC_STOP;
    }
    L.ckpt = true;
  }
};

// ------------------------------------------------------------------------
// Vector-borne disease SEIR model (Section 6.2, Listing 2): one checkpoint per
// day (the `resample` of its `condition`).
//   block 0 (day 0): the parameters from their Beta priors, the initial
//     compartments (hI = 1 + Poisson(5), hE = Poisson(5), hR uniform, mosquitoes
//     n 10^u with u ~ U(-1, 2)), then the condition of day 0;
//   block 1 (day k): humans infected by infectious mosquitoes, exposed, turned
//     infectious and recovered (Binomial draws in the listing's order), the same
//     for mosquitoes, their daily survival (6/7) and births (1/7), then the
//     condition of day k.
// condition: new infectious humans accumulate in z; a report y_k != -1 adds
// log Binomial(y_k | z, rho) to the weight and starts z again from 0.
// PSTATE ints: block index, hS hE hI hR mS mE mI mR z; reals: hLambda hDelta
// hGamma mLambda mDelta rho.  Humans n = 7370.
// ------------------------------------------------------------------------
template <typename Real>
struct SeirModel {
  using R = Real;
  static constexpr int NB = 2, N_REAL = 6, N_INT = 10;
  static constexpr bool HAS_STACK = false;
  struct Lane {
    int pc;
    bool ckpt;
    R logw;
    int overflow, limited;
    int c[9];
    R th[6];
  };
  __device__ static void init(Lane& L) {
    L.pc = 0;
    L.logw = (R)0;
#pragma unroll
    for (int f = 0; f < 9; ++f) L.c[f] = 0;
#pragma unroll
    for (int f = 0; f < 6; ++f) L.th[f] = (R)0;
  }
  __device__ static void gather(Lane& L, const StateView& Sc, const StateView&, int a, int, int N,
                                const ModelDev&) {
    L.pc = Sc.inf_(0, a, N);
#pragma unroll
    for (int f = 0; f < 9; ++f) L.c[f] = Sc.inf_(f + 1, a, N);
#pragma unroll
    for (int f = 0; f < 6; ++f) L.th[f] = Sc.rf<R>(f, a, N);
    L.logw = (R)0;
  }
  __device__ static void store(const Lane& L, const StateView& Sn, int i, int N) {
    Sn.inf_(0, i, N) = L.pc;
#pragma unroll
    for (int f = 0; f < 9; ++f) Sn.inf_(f + 1, i, N) = L.c[f];
#pragma unroll
    for (int f = 0; f < 6; ++f) Sn.rf<R>(f, i, N) = L.th[f];
  }
  __device__ static void load(Lane& L, const StateView&, const SnapView& P, int i, int N,
                              const Stream&) {
    L.pc = P.ints[i];
#pragma unroll
    for (int f = 0; f < 9; ++f) L.c[f] = P.ints[(size_t)(f + 1) * N + i];
#pragma unroll
    for (int f = 0; f < 6; ++f) L.th[f] = (R)P.real[(size_t)f * N + i];
    L.logw = (R)P.logw[i];
  }
  __device__ static void begin(Lane& L) {
    L.ckpt = false;
    L.overflow = L.limited = 0;
  }
  __device__ static void block(int b, Lane& L, Stream& s, const ModelDev& md, const StateView&, int,
                               int k, int) {
    int* C = L.c;
    R* th = L.th;
    int hDeltaI;
    if (b == 0) {
      th[0] = beta_ab<R>(s, (R)1.0, (R)1.0);                                     // hLambda
      th[1] = beta_ab<R>(s, (R)1.0 + (R)2.0 / (R)4.4, (R)3.0 - (R)2.0 / (R)4.4);  // hDelta
      th[2] = beta_ab<R>(s, (R)1.0 + (R)2.0 / (R)4.5, (R)3.0 - (R)2.0 / (R)4.5);  // hGamma
      th[3] = beta_ab<R>(s, (R)1.0, (R)1.0);                                     // mLambda
      th[4] = beta_ab<R>(s, (R)1.0 + (R)2.0 / (R)6.5, (R)3.0 - (R)2.0 / (R)6.5);  // mDelta
      th[5] = beta_ab<R>(s, (R)1.0, (R)1.0);                                     // rho
      const int n = 7370;
      const int hI = 1 + poisson<R>(s, (R)5.0);
      const int hE = poisson<R>(s, (R)5.0);
      const int hR = (int)m_floor(uniform_ab<R>(s, (R)0.0, (R)(n - hI - hE + 1)));
      C[0] = n - hE - hI - hR;
      C[1] = hE;
      C[2] = hI;
      C[3] = hR;
      const R u = uniform_ab<R>(s, (R)-1.0, (R)2.0);
      C[4] = (int)m_floor((R)n * ex(u * (R)2.302585092994045684, s));  // n 10^u
      C[5] = C[6] = C[7] = 0;
      C[8] = 0;
      hDeltaI = hI;
    } else {
      const int hSP = C[0], hEP = C[1], hIP = C[2], hRP = C[3];
      const int mSP = C[4], mEP = C[5], mIP = C[6], mRP = C[7];
      // humans
      const int hN = hSP + hEP + hIP + hRP;
      const int hTau = binomial<R>(s, hSP, (R)1.0 - ex(-((R)mIP / (R)hN), s));
      const int hDeltaE = binomial<R>(s, hTau, th[0]);
      hDeltaI = binomial<R>(s, hEP, th[1]);
      const int hDeltaR = binomial<R>(s, hIP, th[2]);
      C[0] = hSP - hDeltaE;
      C[1] = hEP + hDeltaE - hDeltaI;
      C[2] = hIP + hDeltaI - hDeltaR;
      C[3] = hRP + hDeltaR;
      // mosquitoes
      const int mTau = binomial<R>(s, mSP, (R)1.0 - ex(-((R)hIP / (R)hN), s));
      const int mN = mSP + mEP + mIP + mRP;
      const int mDeltaE = binomial<R>(s, mTau, th[3]);
      const int mDeltaI = binomial<R>(s, mEP, th[4]);
      const int mDeltaR = binomial<R>(s, mIP, (R)0.0);
      int mS = mSP - mDeltaE;
      int mE = mEP + mDeltaE - mDeltaI;
      int mI = mIP + mDeltaI - mDeltaR;
      int mR = mRP + mDeltaR;
      const R mMu = (R)6.0 / (R)7.0, mNu = (R)1.0 / (R)7.0;
      mS = binomial<R>(s, mS, mMu);
      mE = binomial<R>(s, mE, mMu);
      mI = binomial<R>(s, mI, mMu);
      mR = binomial<R>(s, mR, mMu);
      mS = mS + binomial<R>(s, mN, mNu);
      C[4] = mS;
      C[5] = mE;
      C[6] = mI;
      C[7] = mR;
    }
    C[8] = C[8] + hDeltaI;
    const int y = (int)md.obs[k];
    if (y != -1) {
      L.logw = L.logw + binomial_logpmf<R>(y, C[8], th[5], s);
      C[8] = 0;
    }
    L.pc = (k + 1 == md.T) ? PC_STOP : 1;
    L.ckpt = true;
  }
};

// ------------------------------------------------------------------------
// The hidden-lineage frame machine shared by the tree models (Listing 1's
// simBranch / crbdGoesUndetected / iter recursion made explicit): one hidden
// speciation event per call.  The event is the next child of the top frame
// (time ~ U(t - bl, t)) or the branch's next one (~ U(stop, start)); a frame
// whose children all went undetected returns true (at the branch level that
// multiplies the weight by 2: lnProb3 += ln 2).  Then the undetected-lineage
// call at that time: a call deeper than depth_cap, or the (call_limit+1)-th
// call of a segment, kills the particle; the lifetime dur comes from
// M::lifetime; if dur > t the lineage is detected with probability rho (the
// particle dies); the speciation count on min(dur, t) comes from M::count, and
// a positive count pushes a frame.  M::lifetime and M::count take the model's
// draws (and, for delayed sampling, update its posteriors).
// ------------------------------------------------------------------------
template <class M, typename R = typename M::R>
__device__ __forceinline__ void hidden_event(typename M::Lane& L, Stream& s, const ModelDev& md,
                                             int end_block) {
  for (;;) {
    if (L.fsp == 0) {
      if (L.n_top == 0) {
        L.pc = end_block;
        return;
      }
      L.n_top -= 1;
      L.cur_t = uniform_ab<R>(s, L.stop, L.start);
      break;
    }
    const int f = L.fsp - 1;
    if (L.fr_rem[f] == 0) {
      L.fsp = f;
      if (f == 0) L.lnp3 = L.lnp3 + C<R>::ln2;
      continue;
    }
    L.fr_rem[f] -= 1;
    const R t = L.fr_t[f];
    L.cur_t = uniform_ab<R>(s, t - L.fr_bl[f], t);
    break;
  }
  if (L.fsp + 1 > md.depth_cap) {
    L.overflow = 1;
    L.lnp3 = neg_inf<R>();
    L.pc = end_block;
    return;
  }
  L.calls += 1;
  if (L.calls > md.call_limit) {
    L.limited = 1;
    L.lnp3 = neg_inf<R>();
    L.pc = end_block;
    return;
  }
  const R t = L.cur_t;
  const R dur = M::lifetime(L, s);
  if (gt_nonneg(dur, t)) {  // both >= 0
    if (bernoulli<R>(s, (R)md.rho)) {
      L.lnp3 = neg_inf<R>();
      L.pc = end_block;
      return;
    }
  }
  const R bl = dur < t ? dur : t;
  const int j = M::count(L, s, bl);
  if (j == 0) {  // returned true at once
    if (L.fsp == 0) L.lnp3 = L.lnp3 + C<R>::ln2;
    return;
  }
  L.fr_t[L.fsp] = t;
  L.fr_bl[L.fsp] = bl;
  L.fr_rem[L.fsp] = j;
  L.fsp += 1;
}

// ------------------------------------------------------------------------
// Birth-death tree models (Listing 1).  PSTATE crossing checkpoints:
// real 0 = lambda (RATESHIFT: the root rate lambda0), real 1 = mu, int 0 =
// block index; RATESHIFT adds int 1 = stack pointer and the pending-rate
// stack rows.  Segment-local scratch (the hidden-lineage call stack of
// crbdGoesUndetected / iter) never crosses a checkpoint, so it lives in the
// lane's registers and thread-local memory.
//
// Blocks (checkpoints only after 0 and 3):
//   0 PRIOR      lambda ~ Gamma(1, ls), mu ~ Gamma(1, ms); weight(corrFactor)
//   1 BRANCH     simTree body for node v = preorder[k]: lnProb1 = -mu dt,
//                lnProb2 = ln lambda (internal) or ln rho (tip), n ~ Poisson(lambda dt)
//   2 HIDDEN     one hidden speciation event per execution: the next event
//                time (simBranch: ~ U(stop, start); iter of the top frame:
//                ~ U(t - bl, t); finished frames return true first), then the
//                crbdGoesUndetected call at that time: dur ~ Exp(mu); if
//                dur > t, detected with prob rho; j ~ Poisson(lambda min(dur, t));
//                j > 0 pushes a frame
//   3 END        weight(lnProb1 + (lnProb2 + lnProb3)); checkpoint
// A detected hidden lineage makes lnProb3 = -inf and ends the branch at once.
// A call deeper than depth_cap, or the (call_limit+1)-th call of a segment,
// kills the particle (lnProb3 = -inf) and is counted.
// ------------------------------------------------------------------------
template <typename Real, bool RS>
struct TreeModel {
  using R = Real;
  // CRBD keeps log(lambda) as a third, internal real field (computed once at the
  // prior block instead of once per internal-node branch); it is not an output.
  static constexpr int NB = 4, N_REAL = 2, N_INT = RS ? 2 : 1;
  static constexpr bool HAS_STACK = RS;
  enum { PRIOR = 0, BRANCH = 1, HIDDEN = 2, END = 3 };
  struct Lane {
    int pc, sp, v, n_top, fsp, calls;
    bool ckpt, internal;
    int overflow, limited;
    R lam, mu, logw, loglam, inv_mu;
    R lam_b, start, stop, lnp1, lnp2, lnp3, cur_t;
    R fr_t[SMC_MAX_DEPTH], fr_bl[SMC_MAX_DEPTH];
    int fr_rem[SMC_MAX_DEPTH];
  };
  __device__ static void init(Lane& L) {
    L.pc = PRIOR;
    L.sp = 0;
    L.lam = L.mu = L.loglam = (R)0;
    L.logw = (R)0;
  }
  __device__ static void gather(Lane& L, const StateView& Sc, const StateView& Sn, int a, int i,
                                int N, const ModelDev&) {
    L.lam = Sc.rf<R>(0, a, N);
    L.mu = Sc.rf<R>(1, a, N);
    if (!RS) L.loglam = Sc.rf<R>(2, a, N);
    L.pc = Sc.inf_(0, a, N);
    L.logw = (R)0;
    if (RS) {
      // stack-pointer-bounded copy: only rows [0, sp) of the ancestor's stack
      L.sp = Sc.inf_(1, a, N);
      for (int r = 0; r < L.sp; ++r) Sn.st<R>(r, i, N) = Sc.st<R>(r, a, N);
    }
  }
  __device__ static void store(const Lane& L, const StateView& Sn, int i, int N) {
    Sn.rf<R>(0, i, N) = L.lam;
    Sn.rf<R>(1, i, N) = L.mu;
    if (!RS) Sn.rf<R>(2, i, N) = L.loglam;
    Sn.inf_(0, i, N) = L.pc;
    if (RS) Sn.inf_(1, i, N) = L.sp;
  }
  // the snapshot holds lambda and mu; CRBD's internal log(lambda) is formed again
  // exactly as the prior block formed it
  __device__ static void load(Lane& L, const StateView& Sn, const SnapView& P, int i, int N,
                              const Stream& s) {
    L.lam = (R)P.real[i];
    L.mu = (R)P.real[(size_t)N + i];
    L.pc = P.ints[i];
    L.logw = (R)P.logw[i];
    L.sp = 0;
    if (RS) {
      L.sp = P.ints[(size_t)N + i];
      for (int r = 0; r < L.sp; ++r) Sn.st<R>(r, i, N) = (R)P.stack[(size_t)r * N + i];
    } else {
      L.loglam = lg(L.lam, s);
    }
  }
  __device__ static void begin(Lane& L) {
    L.ckpt = false;
    L.overflow = L.limited = 0;
  }
  // hidden_event's draws: a lifetime ~ Exp(mu), a speciation count ~ Poisson(lambda bl)
  __device__ static R lifetime(Lane& L, Stream& s) {
    return L.mu > (R)0 ? exponential_inv(s, L.mu, L.inv_mu) : exponential<R>(s, L.mu);
  }
  __device__ static int count(Lane& L, Stream& s, R bl) { return poisson<R>(s, L.lam_b * bl); }
  __device__ static void block(int b, Lane& L, Stream& s, const ModelDev& md, const StateView& S,
                               int i, int k, int N) {
    switch (b) {
      case PRIOR: {
        if (md.fixed_rates) {
          L.lam = (R)md.lambda_fixed;
          L.mu = (R)md.mu_fixed;
        } else {
          L.lam = gamma1<R>(s, (R)md.lambda_scale);
          L.mu = gamma1<R>(s, (R)md.mu_scale);
        }
        if (RS) {
          S.st<R>(0, i, N) = L.lam;  // the root's rate, pending for its children
          L.sp = 1;
        } else {
          L.loglam = lg(L.lam, s);
        }
        L.logw = L.logw + (R)md.corr;
        L.pc = BRANCH;
        L.ckpt = true;
        return;
      }
      case BRANCH: {
        const BranchRec br = load_branch(md.branch, k);
        const int v = br.v;
        L.v = v;
        L.internal = (br.flags & 1) != 0;
        R lam = L.lam;
        if (RS) {
          R lam_p;
          if (L.sp <= 0) {
            lam_p = L.lam;
          } else if (br.flags & 2) {
            lam_p = S.st<R>(L.sp - 1, i, N);  // left child: parent's rate stays pending
          } else {
            L.sp -= 1;  // right child: last use of the parent's rate
            lam_p = S.st<R>(L.sp, i, N);
          }
          R mult;
          if (md.fixed_mult) {
            mult = (R)md.fixed_mult[v];
          } else {
            Stream sm{s.k0, s.k1, s.n, s.k, 0u, 2u, s.tab};
            mult = lognormal<R>(sm, (R)md.sigma);
          }
          lam = lam_p * mult;
        }
        L.lam_b = lam;
        L.start = (R)br.start;
        L.stop = (R)br.stop;
        const R dt = L.start - L.stop;
        L.lnp1 = -L.mu * dt;
        L.lnp2 = L.internal ? (RS ? lg(lam, s) : L.loglam) : (R)md.log_rho;
        L.n_top = poisson<R>(s, lam * dt);
        if (L.n_top > 0 && L.mu > (R)0) L.inv_mu = (R)1 / L.mu;
        L.lnp3 = (R)0;
        L.fsp = 0;
        L.calls = 0;
        L.pc = HIDDEN;
        return;
      }
      case HIDDEN: {
        hidden_event<TreeModel>(L, s, md, END);
        return;
      }
      default: {  // END
        L.logw = L.logw + (L.lnp1 + (L.lnp2 + L.lnp3));
        if (RS && L.internal) {
          if (L.sp < md.lam_stack_cap) {
            S.st<R>(L.sp, i, N) = L.lam_b;
            L.sp += 1;
          } else {
            L.logw = neg_inf<R>();
            L.overflow += 1;
          }
        }
        L.pc = (k + 1 == md.n_nodes) ? PC_STOP : BRANCH;
        L.ckpt = true;
        return;
      }
    }
  }
};

// ------------------------------------------------------------------------
// CRBD with static delayed sampling (Section 6.3): Listing 1's blocks with
// lambda ~ Gamma(1, lambda_scale) and mu ~ Gamma(1, mu_scale) (shape, scale)
// never drawn; each particle keeps their Gamma(shape, rate) posteriors
// (a_l, b_l) and (a_m, b_m) (real fields 0-3) and every draw that involves a
// rate comes from its predictive law, followed by the conjugate update:
//   0 PRIOR   a_l = 1, b_l = 1/lambda_scale, a_m = 1, b_m = 1/mu_scale;
//             weight(corrFactor); checkpoint
//   1 BRANCH  node v = preorder[k]: lnProb1 = log E[exp(-mu dt)] =
//             -a_m log1p(dt / b_m), b_m += dt; lnProb2 = log E[lambda] =
//             log(a_l / b_l), a_l += 1 (internal) or ln rho (tip);
//             n ~ NegBin(a_l, b_l, dt), a_l += n, b_l += dt
//   2 HIDDEN  one hidden speciation event per execution, as in TreeModel, with
//             dur ~ Lomax(a_m, b_m), a_m += 1, b_m += dur, and
//             j ~ NegBin(a_l, b_l, bl), a_l += j, b_l += bl
//   3 END     weight(lnProb1 + (lnProb2 + lnProb3)); checkpoint
// ------------------------------------------------------------------------
template <typename Real>
struct TreeDsModel {
  using R = Real;
  static constexpr int NB = 4, N_REAL = 4, N_INT = 1;
  static constexpr bool HAS_STACK = false;
  enum { PRIOR = 0, BRANCH = 1, HIDDEN = 2, END = 3 };
  struct Lane {
    int pc, v, n_top, fsp, calls;
    bool ckpt;
    int overflow, limited;
    R al, bl, am, bm, logw;
    R start, stop, lnp1, lnp2, lnp3, cur_t;
    R fr_t[SMC_MAX_DEPTH], fr_bl[SMC_MAX_DEPTH];
    int fr_rem[SMC_MAX_DEPTH];
  };
  __device__ static void init(Lane& L) {
    L.pc = PRIOR;
    L.al = L.bl = L.am = L.bm = (R)0;
    L.logw = (R)0;
  }
  __device__ static void gather(Lane& L, const StateView& Sc, const StateView&, int a, int,
                                int N, const ModelDev&) {
    L.al = Sc.rf<R>(0, a, N);
    L.bl = Sc.rf<R>(1, a, N);
    L.am = Sc.rf<R>(2, a, N);
    L.bm = Sc.rf<R>(3, a, N);
    L.pc = Sc.inf_(0, a, N);
    L.logw = (R)0;
  }
  __device__ static void store(const Lane& L, const StateView& Sn, int i, int N) {
    Sn.rf<R>(0, i, N) = L.al;
    Sn.rf<R>(1, i, N) = L.bl;
    Sn.rf<R>(2, i, N) = L.am;
    Sn.rf<R>(3, i, N) = L.bm;
    Sn.inf_(0, i, N) = L.pc;
  }
  __device__ static void load(Lane& L, const StateView&, const SnapView& P, int i, int N,
                              const Stream&) {
    L.al = (R)P.real[i];
    L.bl = (R)P.real[(size_t)N + i];
    L.am = (R)P.real[(size_t)2 * N + i];
    L.bm = (R)P.real[(size_t)3 * N + i];
    L.pc = P.ints[i];
    L.logw = (R)P.logw[i];
  }
  __device__ static void begin(Lane& L) {
    L.ckpt = false;
    L.overflow = L.limited = 0;
  }
  // hidden_event's draws from the predictive laws, each followed by its
  // conjugate update: a lifetime ~ Lomax(a_m, b_m), then a_m += 1, b_m += dur;
  // a speciation count ~ NegBin(a_l, b_l, bl), then a_l += j, b_l += bl
  __device__ static R lifetime(Lane& L, Stream& s) {
    const R dur = lomax<R>(s, L.am, L.bm);
    L.am = L.am + (R)1.0;
    L.bm = L.bm + dur;
    return dur;
  }
  __device__ static int count(Lane& L, Stream& s, R bl) {
    const int j = neg_binomial<R>(s, L.al, L.bl, bl);
    L.al = L.al + (R)j;
    L.bl = L.bl + bl;
    return j;
  }
  __device__ static void block(int b, Lane& L, Stream& s, const ModelDev& md, const StateView&,
                               int, int k, int) {
    switch (b) {
      case PRIOR: {
        L.al = (R)1.0;
        L.bl = (R)1.0 / (R)md.lambda_scale;
        L.am = (R)1.0;
        L.bm = (R)1.0 / (R)md.mu_scale;
        L.logw = L.logw + (R)md.corr;
        L.pc = BRANCH;
        L.ckpt = true;
        return;
      }
      case BRANCH: {
        const BranchRec br = load_branch(md.branch, k);
        L.v = br.v;
        L.start = (R)br.start;
        L.stop = (R)br.stop;
        const R dt = L.start - L.stop;
        L.lnp1 = -L.am * m_log1p(dt / L.bm);
        L.bm = L.bm + dt;
        if (br.flags & 1) {
          L.lnp2 = lg(L.al / L.bl, s);
          L.al = L.al + (R)1.0;
        } else {
          L.lnp2 = (R)md.log_rho;
        }
        L.n_top = neg_binomial<R>(s, L.al, L.bl, dt);
        L.al = L.al + (R)L.n_top;
        L.bl = L.bl + dt;
        L.lnp3 = (R)0;
        L.fsp = 0;
        L.calls = 0;
        L.pc = HIDDEN;
        return;
      }
      case HIDDEN: {
        hidden_event<TreeDsModel>(L, s, md, END);
        return;
      }
      default: {  // END
        L.logw = L.logw + (L.lnp1 + (L.lnp2 + L.lnp3));
        L.pc = (k + 1 == md.n_nodes) ? PC_STOP : BRANCH;
        L.ckpt = true;
        return;
      }
    }
  }
};

// Per-warp PC-sorted dispatch: while any lane of the warp is still inside
// its segment, pick the block index shared by the most such lanes (ties to
// the larger index) and run that block on exactly those lanes.  The choice
// is warp-uniform, so every block body runs without intra-warp divergence
// on its block index.  Returns the number of blocks this lane executed.
template <class M>
__device__ __forceinline__ int run_segment(typename M::Lane& L, Stream& s, const ModelDev& md,
                                           const StateView& S, int i, int k, int N, bool active) {
  int n_exec = 0;
  if (active) M::begin(L);
  for (;;) {
    const unsigned act = __ballot_sync(0xffffffffu, active);
    if (act == 0u) break;
    int sel;
    if (M::NB == 1) {
      sel = 0;
    } else {
      const unsigned peers = __match_any_sync(0xffffffffu, active ? L.pc : -2);
      const unsigned key = active ? ((unsigned)__popc(peers) << 8) | (unsigned)L.pc : 0u;
      sel = (int)(__reduce_max_sync(0xffffffffu, key) & 0xffu);
    }
    if (active && L.pc == sel) {
      M::block(sel, L, s, md, S, i, k, N);
      n_exec += 1;
      if (L.ckpt) active = false;
    }
  }
  return n_exec;
}

}  // namespace smc
