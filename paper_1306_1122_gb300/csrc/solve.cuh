// solve.cuh -- structures shared by the host driver and the lambda-search kernels.
#pragma once
#include "dbie_internal.cuh"

namespace dbie {

// Per-point simplex state, structure-of-arrays: field f of point g is at [f * N + g].
enum DField {
  D_VL = 0,      // vertex lambda: D_VL + v * 3 + d   (v = 0..3, d = 0..2)
  D_VB = 12,     // vertex field B: D_VB + v * 3 + p
  D_VF = 24,     // vertex f: D_VF + v
  D_VG = 28,     // vertex g
  D_VPHI = 32,   // vertex Phi
  D_RL = 36,     // reflected point: lambda (3), B (3), f, g, Phi
  D_RB = 39,
  D_RF = 42,
  D_RG = 43,
  D_RPHI = 44,
  D_TL = 45,     // pending single trial point lambda (3)
  // certified decisions: the error bound of each value (0 once re-evaluated in float-float)
  D_VS = 48,     // vertex bounds: D_VS + v
  D_RS = 52,     // reflected point's bound
  D_EB = 53,     // evaluated single trial point: B (3), f, g, Phi, bound (kept while its step
  D_EF = 56,     // waits for a float-float re-evaluation)
  D_EG = 57,
  D_EPHI = 58,
  D_ES = 59,
  // certified decisions, difference level: the point's float-float reference value, lambda (3)
  // and its 12 sums (D_REFS = NaN: no reference yet)
  D_REFL = 60,
  D_REFS = 63,
  D_NFIELDS = 75
};
// Quasi-Newton state (same arrays, other meaning): x, grad Phi, inverse Hessian H (3 x 3),
// direction d, B, f, g, Phi at x, line-search step alpha, grad . d, |grad|.
enum BField {
  B_X = 0, B_GR = 3, B_H = 6, B_D = 15, B_B = 18, B_F = 21, B_G = 22, B_PHI = 23, B_ALPHA = 24,
  B_GD = 25, B_GN = 26
};
// I_FLAGS bit F_EVAL: this step's evaluations are in the state (the step waits for a
// re-evaluation); I_RSLOT, I_DSLOT: first float-float and first difference query slot of the
// point's pending re-evaluation; I_RTGT: its targets, one per byte: value id (0..3 vertex,
// 4 reflected point, 5 trial point) | RT_DIF when the value goes to the difference pass,
// 0xff = none.
enum IField { I_STAGE = 0, I_ITERS = 1, I_NFEV = 2, I_STATUS = 3, I_QSLOT = 4, I_FLAGS = 5,
              I_RSLOT = 6, I_RTGT = 7, I_DSLOT = 8, I_NFIELDS = 9 };
constexpr int F_EVAL = 1;
constexpr int RT_DIF = 0x40;
constexpr int VID_R = 4, VID_E = 5;
enum PtStatus { PT_RUNNING = -1, PT_CONVERGED = 0, PT_MAXITER = 1 };
enum Stage { ST_INIT = 0, ST_REFLECT = 1, ST_EXPAND = 2, ST_OCONTRACT = 3, ST_ICONTRACT = 4,
             ST_SHRINK = 5, ST_DONE = 6, ST_BF_INIT = 10, ST_BF_LS = 11 };

struct SolveOpts {
  double eps_f, eps_g, tol, w_g;
  double tie;                // certified decisions: near-tie band factor (0: off)
  int32_t max_iter, dim, near_on, pad0;
  double tie_dif;            // band factor of values re-evaluated by difference (0: level off)
};

// One ping-pong side of the per-round buffers.
struct RoundBuf {
  float4* qpos;        // query slots
  Lam4* qlam;
  int32_t* q_cnt;      // [nprob]
  int32_t* act;        // active points
  int32_t* act_cnt;    // [1]
  int32_t* near;       // near-field query slots
  int32_t* near_cnt;   // [1]
  // certified decisions: float-float re-evaluation queries and the points that wait for them
  float4* fpos;        // [2 N] slots (problem p from its qff_off)
  Lam4* flam;
  int32_t* fq_cnt;     // [nprob]
  int32_t* ref;        // waiting points
  int32_t* ref_cnt;    // [1]
  // difference re-evaluation queries (value lambda, reference lambda; slots as fpos)
  float4* dpos;
  Lam4* dlam;
  Lam4* dlam0;
  int32_t* dq_cnt;     // [nprob]
};

struct SolveArgs {
  const ProbDesc* probs;
  int32_t nprob;
  int32_t pad0;
  int64_t N;                 // total points
  const float4* ppos;        // [N] x, y, z, problem (int bits)
  double* sd;                // [D_NFIELDS * N]
  int32_t* si;               // [I_NFIELDS * N]
  RoundBuf cur, nxt;
  const double* out;         // pair-sum partials of the current round (item chunks)
  const PlanHdr* plan;       // plan of the current round
  const int32_t* item_off;   // [nprob + 1]
  SolveOpts o;
  // final per-point results
  double* res_B;             // [N * 3]
  double* res_lam;           // [N * 3]
  double* res_f;
  double* res_g;
  int32_t* res_iters;
  int32_t* res_status;
  int32_t* res_nfev;
  char* codes;               // [N * codes_stride] or null
  int32_t codes_stride;
  int32_t pad1;
  unsigned* err;
  const double* corr;        // [N * 12] pixel-exact corrections (dB, d grad B), or null
  // certified decisions
  const double* msc;         // [N * 15] sum_k |b_pk| / r^j, j = 1..5, per component (or null)
  const double* msc0;        // [N * 3] sum_k |b_pk| per component (difference level)
  const double* fout;        // float-float pass partial sums of the current round
  const PlanHdr* fplan;
  const int32_t* fitem_off;
  const double* dout;        // difference pass partial sums of the current round
  const PlanHdr* dplan;
  const int32_t* ditem_off;
  unsigned long long* stat_ties;   // near-tie decisions sent to re-evaluation (or null)
  unsigned long long* stat_difs;   // values re-evaluated by difference (or null)
};

struct PlanArgs {
  const ProbDesc* probs;
  int32_t nprob;
  int32_t qper;              // queries per item
  int32_t target_items;
  int32_t nsplit_cap;
  const int32_t* q_cnt_cur;
  int32_t* q_cnt_pass;       // copy of the current counts read by the pair-sum pass
  int32_t* item_off;         // [nprob + 1]
  PlanHdr* plan;
  int32_t* work;
  int32_t* q_cnt_nxt;        // zeroed
  int32_t* act_cnt_nxt;
  int32_t* near_cnt_nxt;
  int32_t* fq_cnt_nxt;       // zeroed (certified decisions; may be null)
  int32_t* dq_cnt_nxt;       // zeroed (difference level; may be null)
  int32_t* ref_cnt_nxt;
  int32_t* round_ctr;        // incremented per round
  unsigned long long* stat_queries;
  double* stat_pairs;
};

}  // namespace dbie
