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
  double r1, r0;        // r of the newest level and of the one before
  double alpha;         // dt r^{n+1} / sqrt(E1) of the pending update
  double zm[2];         // FP64 zero mode of each slot (mean of phi)
  // last SAV solve (diagnostics)
  double E1, S, gamma, eta, theta, denom, LHS, xi;
  // last energy evaluation
  double E_orig, E_mod, E_breve;
  int p, pending, status, pad_;
  long long nsteps;
};

}  // namespace spfc
