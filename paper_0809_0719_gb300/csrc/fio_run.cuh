// fio_run.cuh -- launch shapes and the level schedule of one apply (forward or
// adjoint), templated on precision R and q.  Included once per q by fio_q*.cu.
#pragma once
#include <algorithm>

#include "fio_k32r.cuh"

namespace fio {

// Per-kernel timing with CUDA events recorded on the launch stream around each
// launch (enabled by fio_profile).  Kinds index kKernelNames.
constexpr int kKinds = 10;
constexpr int kProfSlots = 4096;
enum KernelKind {
  K_INIT = 0, K_TRANS_P = 1, K_SWITCH = 2, K_TRANS_X = 3, K_TERM = 4,
  K_TERM_ADJ = 5, K_TRANS_P_ADJ = 6, K_SWITCH_ADJ = 7, K_TRANS_X_ADJ = 8, K_INIT_ADJ = 9
};
static const char *const kKernelNames[kKinds] = {"init", "trans_p", "switch", "trans_x", "term",
                                                 "term_adj", "trans_x_adj", "switch_adj", "trans_p_adj", "init_adj"};
struct Prof {
  int enabled;
  int n;                        // events used
  cudaEvent_t ev[2 * kProfSlots];
  int kind[kProfSlots];
  double ms[kKinds];
  long long launches[kKinds];
};

// Everything a run needs from a plan (plain data, no ownership).
struct PlanDev {
  Tables tb;
  TablesF tf;  // df tables of FIO_F32 plans; tf.xnode == NULL selects the generic kernels
  Phase ph;
  int N, L, q, s, e, l0, lm, l1, precision, nrhs_max, maxsrc, nbox_init;
  void *state[2];
  double T[2][kQMax][kQMax];
  double V[kMMax][kQMax];
  int smem_optin;
  int num_sms;
  int switch_impl;  // FP32 switch: 0 FFMA, 1 tensor cores (A in smem), 2 warp-specialised FFMA,
                    // 3 tensor cores (A in tensor memory), 4 as 3 with two wide MMAs per K-step,
                    // 5 and 6 as 3 and 4 with 3 split-TF32 products instead of 5;
                    // chosen by the plan's autotuner
  int trans_rs;     // FP32 translations of the p-shape (recursion in p, adjoint of the recursion
                    // in x): RHS per subtile 2, 4 or 8, or 32 for the register-tiled kernels
                    // (fio_k32r.cuh, q <= 9); chosen by the plan's autotuner
  int trans_rs_x;   // the same for the x-shape (recursion in x, adjoint of the recursion in p):
                    // 2, 4, 8, or 32 (register-tiled)
  int sw_rb;        // FP32 FFMA switch: RHS per contraction task, 4 or 8 (chosen by the plan's autotuner)
  int *status;  // device status word: 1 = a bounded wait expired (read by fio_check)
  unsigned long long handoff_ns;  // tensor-memory switch: limit of its hand-off waits (0 = normal; tests)
  Prof *prof;   // NULL unless profiling was ever enabled
};

enum RunKind { RUN_FWD = 0, RUN_ADJ = 1, RUN_COUNT_FWD = 2, RUN_COUNT_ADJ = 3, RUN_TUNE = 4, RUN_TC_OK = 5 };

constexpr int kSmemTarget = 100 * 1024;  // per-CTA budget of the translation kernels

template <typename K> static cudaError_t set_smem(K kernel, int optin) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

template <typename R, int Q> struct Runner {
  typedef typename C2<R>::T CT;
  static constexpr int Q2 = Q * Q;
  const PlanDev &p;
  cudaStream_t st;
  int nrhs;
  bool count_only;
  int launches = 0;

  Runner(const PlanDev &pp, cudaStream_t s, int n, bool c) : p(pp), st(s), nrhs(n), count_only(c) {}

  Geom geom(int l, int rt, int U, long long nunits) const {
    Geom g;
    g.L = p.L;
    g.e = p.e;
    g.q = Q;
    g.s = p.s;
    g.l = l;
    g.nrhs = nrhs;
    g.rt = rt;
    g.U = U;
    g.nunits = nunits;
    return g;
  }
  TMat<R, Q> tmat() const {
    TMat<R, Q> t;
    for (int s = 0; s < 2; s++)
      for (int i = 0; i < Q; i++)
        for (int j = 0; j < Q; j++) t.T[s][i][j] = (R)p.T[s][i][j];
    return t;
  }
  VMat<R, Q> vmat() const {
    VMat<R, Q> v;
    for (int m = 0; m < kMMax; m++)
      for (int j = 0; j < Q; j++) v.V[m][j] = (R)p.V[m][j];
    return v;
  }
  long long nb_at(int lb) const { return (1LL << lb) << (lb + p.e); }

  int slot = -1;
  void pre(int kind) {
    slot = -1;
    Prof *pr = p.prof;
    if (count_only || !pr || !pr->enabled || pr->n >= kProfSlots) return;
    slot = pr->n++;
    pr->kind[slot] = kind;
    cudaEventRecord(pr->ev[2 * slot], st);
  }
  int check() {
    launches++;
    if (count_only) return 0;
    if (slot >= 0) cudaEventRecord(p.prof->ev[2 * slot + 1], st);
    cudaError_t err = cudaGetLastError();
    return err == cudaSuccess ? 0 : (int)err;
  }

  bool fast32() const { return sizeof(R) == 4 && p.tf.xnode != nullptr; }

  template <bool TYPE_P, bool FWD, int RS> int trans32(int l, const CT *in, CT *out) {
    const long long nunits = (1LL << (2 * (l - 1))) * nb_at(p.L - l);
    const Geom g = geom(l, kRMax, 1, nunits);
    dim3 grid((unsigned)nunits, (unsigned)((nrhs + kRMax - 1) / kRMax));
    if (count_only) return check();
    pre(TYPE_P ? (FWD ? K_TRANS_P : K_TRANS_P_ADJ) : (FWD ? K_TRANS_X : K_TRANS_X_ADJ));
    auto k = k32_trans<Q, TYPE_P, FWD, RS>;
    set_smem(k, p.smem_optin);
    k<<<grid, TransShape<Q, RS>::threads, TransShape<Q, RS>::smem, st>>>(p.tb, p.tf, p.ph, g, tmat(),
                                                                         (const float2 *)in, (float2 *)out);
    return check();
  }

  // Register-tiled translation (32 RHS per CTA, one per lane).
  template <bool TYPE_P, bool FWD> int trans32r(int l, const CT *in, CT *out) {
    if constexpr (Q <= 9) {
      const long long nunits = (1LL << (2 * (l - 1))) * nb_at(p.L - l);
      const Geom g = geom(l, kRT, 1, nunits);
      dim3 grid((unsigned)nunits, (unsigned)((nrhs + kRT - 1) / kRT));
      if (count_only) return check();
      pre(TYPE_P ? (FWD ? K_TRANS_P : K_TRANS_P_ADJ) : (FWD ? K_TRANS_X : K_TRANS_X_ADJ));
      if (TYPE_P) {
        auto k = k32_trans_rp<Q, FWD>;
        set_smem(k, p.smem_optin);
        k<<<grid, 4 * kRT, trans_rp_smem_bytes(Q), st>>>(p.tb, p.tf, p.ph, g, tmat(), (const float2 *)in, (float2 *)out,
                                                        p.status);
      } else {
        auto k = k32_trans_rx<Q, FWD>;
        set_smem(k, p.smem_optin);
        k<<<grid, 4 * kRT, trans_rx_smem_bytes(Q), st>>>(p.tb, p.tf, p.ph, g, tmat(), (const float2 *)in, (float2 *)out,
                                                        p.status);
      }
      return check();
    }
    return (int)cudaErrorInvalidConfiguration;
  }
  bool trans_r_ok() const {
    return fast32() && Q <= 9 && p.status && trans_rp_smem_bytes(Q) <= p.smem_optin &&
           trans_rx_smem_bytes(Q) <= p.smem_optin;
  }

  // Translation at level l (forward: l-1 -> l; adjoint: l -> l-1).
  template <bool TYPE_P, bool FWD> int trans(int l, const CT *in, CT *out) {
    if constexpr (sizeof(R) == 4) {
      if (fast32()) {
        const int rs = TYPE_P ? p.trans_rs : p.trans_rs_x;
        if (rs == 32 && trans_r_ok()) return trans32r<TYPE_P, FWD>(l, in, out);
        if (rs == 2) return trans32<TYPE_P, FWD, 2>(l, in, out);
        if (rs == 4) return trans32<TYPE_P, FWD, 4>(l, in, out);
        return trans32<TYPE_P, FWD, 8>(l, in, out);
      }
    }
    const int rt = std::min(nrhs, sizeof(R) == 4 ? 8 : 4);
    const int per_unit = (12 * rt * Q2 + 20 * Q2) * (int)sizeof(CT);
    int U = std::max(1, (64 + rt * Q - 1) / (rt * Q));
    U = std::max(1, std::min(U, kSmemTarget / per_unit));
    const long long nunits = (1LL << (2 * (l - 1))) * nb_at(p.L - l);
    const Geom g = geom(l, rt, U, nunits);
    dim3 grid((unsigned)((nunits + U - 1) / U), (unsigned)((nrhs + rt - 1) / rt));
    const int smem = U * per_unit;
    if (count_only) return check();
    pre(TYPE_P ? (FWD ? K_TRANS_P : K_TRANS_P_ADJ) : (FWD ? K_TRANS_X : K_TRANS_X_ADJ));
    if (TYPE_P) {
      auto k = k_trans_p<R, Q, FWD>;
      set_smem(k, p.smem_optin);
      k<<<grid, kThreads, smem, st>>>(p.tb, p.ph, g, tmat(), in, out);
    } else {
      auto k = k_trans_x<R, Q, FWD>;
      set_smem(k, p.smem_optin);
      k<<<grid, kThreads, smem, st>>>(p.tb, p.ph, g, tmat(), in, out);
    }
    return check();
  }

  static size_t tm_smem(int v) {
    return v == 0 ? TmShape<Q, false, 5>::smem_bytes()
         : v == 1 ? TmShape<Q, true, 5>::smem_bytes()
         : v == 2 ? TmShape<Q, false, 3>::smem_bytes()
                  : TmShape<Q, true, 3>::smem_bytes();
  }
  template <bool FWD> int sw(const CT *in, CT *out) {
    if constexpr (sizeof(R) == 4) {
      if (fast32() && p.switch_impl == 2 && SwWs<Q>::smem <= p.smem_optin) {
        const long long pairs = (1LL << (2 * p.lm)) * nb_at(p.L - p.lm);
        const long long nwork = pairs * ((nrhs + kRMax - 1) / kRMax);
        const Geom g = geom(p.lm, kRMax, 1, pairs);
        const unsigned grid = (unsigned)std::min<long long>(nwork, std::max(1, p.num_sms));
        if (count_only) return check();
        pre(FWD ? K_SWITCH : K_SWITCH_ADJ);
        auto k = k32_switch_ws<Q, FWD>;
        set_smem(k, p.smem_optin);
        k<<<grid, SwWs<Q>::threads, SwWs<Q>::smem, st>>>(p.tb, p.tf, p.ph, g, (const float2 *)in, (float2 *)out, nwork);
        return check();
      }
      // 3 / 4: narrow / wide MMAs with 5 split-TF32 products; 5 / 6: the same with 3
      const int tmv = p.switch_impl - 3;
      const size_t smem_tm = tm_smem(tmv);
      if (fast32() && tmv >= 0 && tmv < 4 && p.status && smem_tm <= (size_t)p.smem_optin) {
        const long long pairs = (1LL << (2 * p.lm)) * nb_at(p.L - p.lm);
        const Geom g = geom(p.lm, kRMax, 1, pairs);
        const long long nsu = pairs >> (p.L - p.lm);  // (box A, angular box) super-units
        dim3 grid((unsigned)std::min<long long>(nsu, std::max(1, p.num_sms)), (unsigned)((nrhs + kRMax - 1) / kRMax));
        if (count_only) return check();
        pre(FWD ? K_SWITCH : K_SWITCH_ADJ);
        auto k = tmv == 0 ? k32_switch_tm<Q, FWD, false, 5>
                 : tmv == 1 ? k32_switch_tm<Q, FWD, true, 5>
                 : tmv == 2 ? k32_switch_tm<Q, FWD, false, 3>
                            : k32_switch_tm<Q, FWD, true, 3>;
        set_smem(k, p.smem_optin);
        k<<<grid, kTmThreads, smem_tm, st>>>(p.tb, p.tf, p.ph, g, (const float2 *)in, (float2 *)out, p.status,
                                             p.handoff_ns);
        return check();
      }
      const size_t smem_tc = TcShape<Q>::smem_bytes();
      if (fast32() && p.switch_impl == 1 && p.status && smem_tc <= (size_t)p.smem_optin) {
        const long long pairs = (1LL << (2 * p.lm)) * nb_at(p.L - p.lm);
        const Geom g = geom(p.lm, kRMax, 1, pairs);
        dim3 grid((unsigned)std::min<long long>(pairs, 2LL * std::max(1, p.num_sms)), (unsigned)((nrhs + kRMax - 1) / kRMax));
        if (count_only) return check();
        pre(FWD ? K_SWITCH : K_SWITCH_ADJ);
        auto k = k32_switch_tc<Q, FWD>;
        set_smem(k, p.smem_optin);
        k<<<grid, kTcThreads, smem_tc, st>>>(p.tb, p.tf, p.ph, g, (const float2 *)in, (float2 *)out, p.status);
        return check();
      }
      const int smem32 = sw32_smem_bytes(Q);
      if (fast32() && smem32 <= p.smem_optin) {
        const long long pairs = (1LL << (2 * p.lm)) * nb_at(p.L - p.lm);
        const Geom g = geom(p.lm, kRMax, 1, pairs);
        dim3 grid((unsigned)pairs, (unsigned)((nrhs + kRMax - 1) / kRMax));
        if (count_only) return check();
        pre(FWD ? K_SWITCH : K_SWITCH_ADJ);
        auto k = p.sw_rb == 8 ? k32_switch<Q, FWD, 8> : k32_switch<Q, FWD, 4>;
        set_smem(k, p.smem_optin);
        k<<<grid, SwShape<Q>::threads, smem32, st>>>(p.tb, p.tf, p.ph, g, (const float2 *)in, (float2 *)out);
        return check();
      }
    }
    const int rt = std::min(nrhs, 32);
    const long long pairs = (1LL << (2 * p.lm)) * nb_at(p.L - p.lm);
    int U = 1;
    if (rt * Q2 < 1024) U = std::max(1, std::min(8, 1024 / (rt * Q2)));
    const int kbudget = 64 * 1024;
    int TC = std::max(1, std::min(Q2, kbudget / (U * Q2 * (int)sizeof(CT))));
    const int smem = (U * rt * Q2 + U * TC * Q2) * (int)sizeof(CT);
    const Geom g = geom(p.lm, rt, U, pairs);
    dim3 grid((unsigned)((pairs + U - 1) / U), (unsigned)((nrhs + rt - 1) / rt));
    if (count_only) return check();
    pre(FWD ? K_SWITCH : K_SWITCH_ADJ);
    auto k = k_switch<R, Q, FWD>;
    set_smem(k, p.smem_optin);
    k<<<grid, kThreads, smem, st>>>(p.tb, p.ph, g, TC, in, out);
    return check();
  }

  int init(const CT *f, CT *out) {
    const int ms = std::max(1, p.maxsrc);
    if constexpr (sizeof(R) == 4) {
      if (fast32()) {
        int GA = std::min(kInitChunk, 1 << (2 * p.l0));
        // with 32 or more RHS: room for one staged output block (kRMax q^2 complex, 16-byte aligned)
        int use_stage = nrhs >= kRMax ? 1 : 0;
        auto bytes = [&](int ga) {
          return (ms * kRMax + ga * ms + ga * Q2) * 8 + ms * 2 * Q * 4 + ga * ((int)sizeof(XDesc) + Q * 8) +
                 (use_stage ? 16 + kRMax * Q2 * 8 : 0);
        };
        while (bytes(GA) > p.smem_optin && GA > 1) GA--;
        if (bytes(GA) > p.smem_optin && use_stage) {
          use_stage = 0;
          GA = std::min(kInitChunk, 1 << (2 * p.l0));
          while (bytes(GA) > p.smem_optin && GA > 1) GA--;
        }
        if (bytes(GA) <= p.smem_optin) {
          const Geom g = geom(p.l0, kRMax, 1, p.nbox_init);
          dim3 grid((unsigned)p.nbox_init, (unsigned)((nrhs + kRMax - 1) / kRMax));
          if (count_only) return check();
          pre(K_INIT);
          auto k = k32_init<Q>;
          set_smem(k, p.smem_optin);
          k<<<grid, InitShape<Q>::threads, bytes(GA), st>>>(p.tb, p.tf, p.ph, g, ms, GA, (const float2 *)f,
                                                             (float2 *)out, use_stage);
          return check();
        }
      }
    }
    int rt = std::min(nrhs, sizeof(R) == 4 ? 32 : 8);
    int GA = std::max(1, kThreads / (rt * Q));
    auto bytes = [&](int rt_, int ga) {
      return (ms * rt_ + ga * ms + ga * Q2) * (int)sizeof(CT) + ms * 2 * Q * (int)sizeof(R);
    };
    while (bytes(rt, GA) > p.smem_optin && GA > 1) GA--;
    while (bytes(rt, GA) > p.smem_optin && rt > 1) rt--;
    if (bytes(rt, GA) > p.smem_optin) return (int)cudaErrorInvalidConfiguration;
    const Geom g = geom(p.l0, rt, 1, p.nbox_init);
    dim3 grid((unsigned)p.nbox_init, (unsigned)((nrhs + rt - 1) / rt));
    if (count_only) return check();
    pre(K_INIT);
    auto k = k_init<R, Q>;
    set_smem(k, p.smem_optin);
    k<<<grid, kThreads, bytes(rt, GA), st>>>(p.tb, p.ph, g, ms, GA, f, out);
    return check();
  }

  int init_adj(const CT *in, CT *fbar) {
    const int ms = std::max(1, p.maxsrc);
    if constexpr (sizeof(R) == 4) {
      const int b32 = (ms * kRMax + ms + Q2 + kRMax * Q2) * 8 + ms * 2 * Q * 4;
      if (fast32() && b32 <= p.smem_optin) {
        const Geom g = geom(p.l0, kRMax, 1, p.nbox_init);
        dim3 grid((unsigned)p.nbox_init, (unsigned)((nrhs + kRMax - 1) / kRMax));
        if (count_only) return check();
        pre(K_INIT_ADJ);
        auto k = k32_init_adj<Q>;
        set_smem(k, p.smem_optin);
        k<<<grid, 256, b32, st>>>(p.tb, p.tf, p.ph, g, ms, (const float2 *)in, (float2 *)fbar);
        return check();
      }
    }
    int rt = std::min(nrhs, sizeof(R) == 4 ? 32 : 8);
    auto bytes = [&](int rt_) {
      return (ms * rt_ + ms + Q2 + rt_ * Q2) * (int)sizeof(CT) + ms * 2 * Q * (int)sizeof(R);
    };
    while (bytes(rt) > p.smem_optin && rt > 1) rt--;
    if (bytes(rt) > p.smem_optin) return (int)cudaErrorInvalidConfiguration;
    const Geom g = geom(p.l0, rt, 1, p.nbox_init);
    dim3 grid((unsigned)p.nbox_init, (unsigned)((nrhs + rt - 1) / rt));
    if (count_only) return check();
    pre(K_INIT_ADJ);
    auto k = k_init_adj<R, Q>;
    set_smem(k, p.smem_optin);
    k<<<grid, kThreads, bytes(rt), st>>>(p.tb, p.ph, g, ms, in, fbar);
    return check();
  }

  int term(const CT *in, CT *u) {
    const int M = 1 << p.s, M2 = M * M;
    if constexpr (sizeof(R) == 4) {
      const int b32 = (2 * kRMax * Q2 + kRMax * kTermM * Q + 2 * (Q2 + kTermM * kTermM)) * 8 +
                      (Q2 + M2) * (int)sizeof(XDesc);
      if (fast32() && M <= kTermM && b32 <= p.smem_optin) {
        const long long nA = 1LL << (2 * p.l1);
        const Geom g = geom(p.l1, kRMax, 1, nA);
        dim3 grid((unsigned)nA, (unsigned)((nrhs + kRMax - 1) / kRMax));
        if (count_only) return check();
        pre(K_TERM);
        auto k = k32_term<Q>;
        set_smem(k, p.smem_optin);
        k<<<grid, 32 * std::max(Q, kTermM), b32, st>>>(p.tb, p.tf, p.ph, g, vmat(), (const float2 *)in, (float2 *)u);
        return check();
      }
    }
    int rt = std::min(nrhs, sizeof(R) == 4 ? 32 : 8);
    auto bytes = [&](int rt_) { return (rt_ * M2 + Q2 + M2 + rt_ * Q2 + rt_ * M * Q) * (int)sizeof(CT); };
    while (bytes(rt) > p.smem_optin && rt > 1) rt--;
    if (bytes(rt) > p.smem_optin) return (int)cudaErrorInvalidConfiguration;
    const long long nA = 1LL << (2 * p.l1);
    const Geom g = geom(p.l1, rt, 1, nA);
    dim3 grid((unsigned)nA, (unsigned)((nrhs + rt - 1) / rt));
    if (count_only) return check();
    pre(K_TERM);
    auto k = k_term<R, Q>;
    set_smem(k, p.smem_optin);
    k<<<grid, kThreads, bytes(rt), st>>>(p.tb, p.ph, g, vmat(), in, u);
    return check();
  }

  int term_adj(const CT *g_in, CT *out) {
    const int M = 1 << p.s, M2 = M * M;
    if constexpr (sizeof(R) == 4) {
      const int b32 = (kRMax * kTermM * kTermM + kRMax * Q * kTermM + kTermM * kTermM + Q2) * 8 +
                      (Q2 + M2) * (int)sizeof(XDesc);
      if (fast32() && M <= kTermM && b32 <= p.smem_optin) {
        const long long nA = 1LL << (2 * p.l1);
        const Geom g = geom(p.l1, kRMax, 1, nA);
        dim3 grid((unsigned)nA, (unsigned)((nrhs + kRMax - 1) / kRMax));
        if (count_only) return check();
        pre(K_TERM_ADJ);
        auto k = k32_term_adj<Q>;
        set_smem(k, p.smem_optin);
        k<<<grid, 32 * std::max(Q, kTermM), b32, st>>>(p.tb, p.tf, p.ph, g, vmat(), (const float2 *)g_in,
                                                       (float2 *)out);
        return check();
      }
    }
    int rt = std::min(nrhs, sizeof(R) == 4 ? 32 : 8);
    auto bytes = [&](int rt_) { return (2 * rt_ * M2 + M2 + Q2 + rt_ * Q * M) * (int)sizeof(CT); };
    while (bytes(rt) > p.smem_optin && rt > 1) rt--;
    if (bytes(rt) > p.smem_optin) return (int)cudaErrorInvalidConfiguration;
    const long long nA = 1LL << (2 * p.l1);
    const Geom g = geom(p.l1, rt, 1, nA);
    dim3 grid((unsigned)nA, (unsigned)((nrhs + rt - 1) / rt));
    if (count_only) return check();
    pre(K_TERM_ADJ);
    auto k = k_term_adj<R, Q>;
    set_smem(k, p.smem_optin);
    k<<<grid, kThreads, bytes(rt), st>>>(p.tb, p.ph, g, vmat(), g_in, out);
    return check();
  }

  // Autotuner: time the alternatives on the plan's state buffers (their contents do
  // not matter) and keep the fastest: the switch implementations of switch_impls(), and
  // the RHS subtile width or register-tiled kernels of each translation shape.  Returns
  // the chosen switch implementation.
  // Bit i set: switch implementation i can run this plan (0 FFMA, 1 tensor cores with
  // the kernel matrix in shared memory, 2 warp-specialised FFMA, 3-6 tensor cores with
  // the kernel matrix in tensor memory: narrow or wide MMAs, 5 or 3 products).
  int switch_impls() const {
    if constexpr (sizeof(R) != 4) {
      return 1;
    } else {
      if (!fast32()) return 1;
      int m = 1;
      if (p.status && TcShape<Q>::smem_bytes() <= (size_t)p.smem_optin) m |= 2;
      if (SwWs<Q>::smem <= p.smem_optin) m |= 4;
      for (int v = 0; v < 4; v++)
        if (p.status && tm_smem(v) <= (size_t)p.smem_optin && (1 << (p.L - p.lm)) <= kTmNb1Max) m |= 8 << v;
      return m;
    }
  }
  template <typename F> float best_ms(F &&fn) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int rep = 0; rep < 3; rep++) {
      cudaEventRecord(a, st);
      fn();
      cudaEventRecord(b, st);
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      if (rep > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
  }
  int tune_switch(PlanDev &pm) {
    if constexpr (sizeof(R) != 4) {
      return 0;
    } else {
      if (!fast32()) return 0;
      const CT *s0 = (const CT *)p.state[0];
      CT *s1 = (CT *)p.state[1];
      if (p.l1 > p.l0) {  // translation kernels: RHS subtile width or the register-tiled kernels,
        // for each shape on its own (timed on a forward level of that shape if the plan has
        // one, else on the adjoint level that uses it)
        const bool has_p = p.lm > p.l0, has_x = p.l1 > p.lm;
        for (int shape = 0; shape < 2; shape++) {
          float best = 1e30f;
          int pick = 8;
          for (int rs : {2, 4, 8, 32}) {
            if (rs == 32 && !trans_r_ok()) continue;
            int &field = shape == 0 ? pm.trans_rs : pm.trans_rs_x;
            field = rs;
            float ms;
            if (shape == 0)
              ms = has_p ? best_ms([&]() { trans<true, true>(p.l0 + 1, s0, s1); })
                         : best_ms([&]() { trans<true, false>(p.lm + 1, s0, s1); });
            else
              ms = has_x ? best_ms([&]() { trans<false, true>(p.lm + 1, s0, s1); })
                         : best_ms([&]() { trans<false, false>(p.l0 + 1, s0, s1); });
            if (ms < best) {
              best = ms;
              pick = rs;
            }
          }
          (shape == 0 ? pm.trans_rs : pm.trans_rs_x) = pick;
        }
      }
      const int avail = switch_impls();
      float best = 1e30f;
      int pick = 0, pick_rb = 4;
      for (int impl = 0; impl < 7; impl++) {
        if (!(avail >> impl & 1)) continue;
        for (int rb : {4, 8}) {
          if (impl != 0 && rb != 4) continue;  // only the one-pair-per-CTA kernel has both tiles
          pm.switch_impl = impl;
          pm.sw_rb = rb;
          const float ms = best_ms([&]() { sw<true>(s0, s1); });
          if (ms < best) {
            best = ms;
            pick = impl;
            pick_rb = rb;
          }
        }
      }
      pm.switch_impl = pick;
      pm.sw_rb = pick_rb;
      return pick;
    }
  }

  // Forward apply; stop_stage >= 0 stops after that stage and leaves its state in *stage_out.
  int forward(const void *f, void *u, int stop_stage, const void **stage_out) {
    CT *S[2] = {(CT *)p.state[0], (CT *)p.state[1]};
    int cur = 0, stage = 0, rc;
    if ((rc = init((const CT *)f, S[cur]))) return rc;
    if (stop_stage == stage) return *stage_out = S[cur], 0;
    for (int l = p.l0 + 1; l <= p.lm; l++) {
      if ((rc = trans<true, true>(l, S[cur], S[cur ^ 1]))) return rc;
      cur ^= 1;
      if (stop_stage == ++stage) return *stage_out = S[cur], 0;
    }
    if ((rc = sw<true>(S[cur], S[cur ^ 1]))) return rc;
    cur ^= 1;
    if (stop_stage == ++stage) return *stage_out = S[cur], 0;
    for (int l = p.lm + 1; l <= p.l1; l++) {
      if ((rc = trans<false, true>(l, S[cur], S[cur ^ 1]))) return rc;
      cur ^= 1;
      if (stop_stage == ++stage) return *stage_out = S[cur], 0;
    }
    return term(S[cur], (CT *)u);
  }

  // Adjoint apply: the forward steps conjugate-transposed, in reverse order.
  int adjoint(const void *g, void *fbar) {
    CT *S[2] = {(CT *)p.state[0], (CT *)p.state[1]};
    int cur = 0, rc;
    if ((rc = term_adj((const CT *)g, S[cur]))) return rc;
    for (int l = p.l1; l >= p.lm + 1; l--) {
      if ((rc = trans<true, false>(l, S[cur], S[cur ^ 1]))) return rc;
      cur ^= 1;
    }
    if ((rc = sw<false>(S[cur], S[cur ^ 1]))) return rc;
    cur ^= 1;
    for (int l = p.lm; l >= p.l0 + 1; l--) {
      if ((rc = trans<false, false>(l, S[cur], S[cur ^ 1]))) return rc;
      cur ^= 1;
    }
    return init_adj(S[cur], (CT *)fbar);
  }
};

// Widen one stage snapshot to complex128 in canonical order (RHS 0 of an nrhs=1 run).
template <typename V> __global__ void k_to_c128(const V *__restrict__ in, double2 *__restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = make_double2((double)in[i].x, (double)in[i].y);
}

template <typename R, int Q>
int run_plan(const PlanDev &p, int kind, const void *in, void *out, int nrhs, cudaStream_t st, int stop_stage,
             int *launches) {
  const bool count = kind == RUN_COUNT_FWD || kind == RUN_COUNT_ADJ;
  Runner<R, Q> r(p, st, nrhs, count);
  int rc;
  if (kind == RUN_TC_OK) {  // which switch implementations can this plan use (bit mask)?
    if (launches) *launches = r.switch_impls();
    return 0;
  }
  if (kind == RUN_TUNE) {
    const int impl = r.tune_switch(const_cast<PlanDev &>(p));
    if (launches) *launches = impl;
    return (int)cudaGetLastError();
  }
  if (kind == RUN_FWD || kind == RUN_COUNT_FWD) {
    const void *snap = nullptr;
    rc = r.forward(in, out, stop_stage, &snap);
    if (rc == 0 && stop_stage >= 0 && !count) {
      const long long n = ((long long)p.N * p.N * Q * Q) << p.e;
      k_to_c128<typename C2<R>::T><<<592, 256, 0, st>>>((const typename C2<R>::T *)snap, (double2 *)out, n);
      rc = (int)cudaGetLastError();
    }
  } else {
    rc = r.adjoint(in, out);
  }
  if (launches) *launches = r.launches;
  return rc;
}

}  // namespace fio
