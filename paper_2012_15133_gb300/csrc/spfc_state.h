// Per-run parameters and the device-resident SAV scalar record.
#pragma once

#include <stdint.h>

namespace spfc {

// Constant per run (rebuilt when dt changes). All quantities follow the
// paper's notation on a box [0,L]^d with N points per axis.
struct Params {
  int d;          // 2 or 3
  int N;          // points per axis
  int NH;         // N/2 + 1 (half-spectrum length along x)
  double kf[3];   // 2 pi / L per axis (x, y, z)
  double hd;      // h^d in <f,g> = h^d sum f g
  double vol;     // |Omega|
  double P;       // number of grid points N^d
  double a;       // 1 - eps
  double beta;    // coefficient of 1/4 |grad phi|^4
  double C;       // C_beta = 1 + 1/beta (E_1 >= |Omega|)
  double dt;
  double invP;    // 1 / P
  // float32 copies for the float32-bulk kernels (no float64 work per thread)
  float kf_f[3];
  float dt_f, a_f, beta_f, invP_f;
  // stabiliser of Sec. 5.2 (- A dt Delta_N (phi^{n+1} - phi^n)); A = 0: the scheme of Sec. 2
  double stab;    // A
  double sdt;     // A dt
  float sdt_f;
  // optional phi^4 term: E_1 gains gamma3/4 ||phi||_4^4 and N gains gamma3 phi^3
  // with its mean removed (2D single runs); gamma3 = 0 is the SPFC model
  double g3;      // gamma3
  double g3b;     // gamma3 / beta (folded into the sum of s^2 that E_1 takes with beta/4)
  float g3_f, g3b_f;
  // model: 0 the SPFC equation (the paper's), 1 the PFC model of Sec. 1
  // (eq. energy-PFC; g3 is its phi^4 coefficient, beta unused), with the
  // split L = a + (1 + Delta)^2, E_1 = g3/4 ||phi||_4^4 - 1/2 ||phi||^2 + C |Omega|
  int pfc;
  // E_1 = hd (e1c4 q0 + e1c2 q1) + C |Omega| from the row pass's sums q0, q1
  // (SPFC: sum s^2 and sum s with beta/4 and -1; PFC: sum phi^4 and sum phi^2
  // with g3/4 and -1/2)
  double e1c4, e1c2;
  // the box lengths and eps exactly as given at creation (kf and a derive from them)
  double Lbox[3];
  double eps;
};

enum PendingKind : int { PEND_NONE = 0, PEND_BDF2 = 1, PEND_BDF1 = 2 };

// Device status codes (mirrors spfc_status of the C interface)
enum DevStatus : int { DEV_OK = 0, DEV_NONFINITE = 4, DEV_TIMEOUT = 5 };

// Device-resident scalar state of one run. Slot p of the two spectral state
// buffers holds the newest level phi^n, slot 1-p the previous one. When
// `pending` is set, phi^{n+1} = alpha * b + c is known implicitly through the
// stored N_hat and is materialised by the next step's first kernel (or by an
// explicit finalize), which also flips p.
struct SavScal {
  double r1, r0;        // r of the newest level and of the one before (float64 on both paths)
  double alpha;         // dt r^{n+1} / sqrt(E1) of the pending update
  float alpha_f;        // the same, rounded to float32 (read by float32-bulk kernels)
  int pad0_;
  double zm[2];         // FP64 zero mode of each slot (mean of phi)
  // last SAV solve (diagnostics)
  double E1, S, gamma, eta, theta, denom, LHS, xi;
  // last energy evaluation
  double E_orig, E_mod, E_breve;
  int p, pending, status, pad_;
  long long nsteps;
  // optional per-step record ring in pinned host memory (device-visible
  // pointer; NULL: none): every committed solve writes kRingFields doubles
  // {steps, r^{n+1}, r^n, xi, gamma, E_1, alpha, status} at entry steps % cap.
  double* ring;
  long long ring_cap;
};
constexpr int kRingFields = 8;

}  // namespace spfc
