// Device-resident solver state shared by the host API and the kernels.
//
// One FistaState lives in device memory per solve.  The kernels read it at
// the start of every pass (momentum factor, step, which iterate buffer is
// current, whether the run is finished) and the fold kernel's last block
// updates it after every pass, so a captured CUDA graph of many passes needs
// no host round trip.  Iterate Xbar^j lives in buffer j & 1.
#pragma once
#include <stdint.h>

namespace fc {

struct FistaState {
  // scalars in float64
  double S2;          // ||S||_F^2
  double tau;         // step size
  double L;           // Lipschitz bound used for tau (0 for a constant step)
  double tol;         // stopping tolerance
  double t;           // t_n of the pass about to run (t_1 = 1)
  double beta;        // momentum factor (t_{n-1} - 1) / t_n of the pass about to run
  double beta_next;   // momentum factor of the pass after it (forms Y^{n+1} one pass early)
  double gram2_cur;   // ||Xbar^{pass}^T Xbar^{pass}||_F^2
  double loss_prev;   // newest known loss before loss_last (stop test)
  double loss_last;   // f(Xbar^{f_iter})
  double trace_last;  // sum_i <x_i, (S X)_i> of Xbar^{f_iter}
  double gram2_last;  // ||Gram||_F^2 of Xbar^{f_iter}
  double pg_first;    // r_1
  double pg_last;     // newest r_n
  double shift;       // mean entry subtracted from the Gram of Y before the float32 round
  // counters
  int64_t pass;       // passes completed = index of the newest iterate
  int64_t limit;      // passes allowed so far (set by the host per call)
  int64_t max_iter;
  int64_t f_iter;     // -1 until a loss is known
  int64_t out_iter;   // iterate cluster_get_U returns
  int32_t done;
  int32_t status;     // 0 ok, 4 nonfinite, 5 max_iter, 6 a bounded wait gave up
  int32_t stop_rule;
  int32_t accel;
  int32_t k;
  uint32_t ticket;    // block counter of the fold kernel (reset by its last block)
  int32_t eval_mode;
  int32_t hooks;      // test hooks (cluster_test_hooks); 0 in normal operation
  double eval_f;      // result of the last objective-only pass
  double eval_trace;
  double eval_gram2;
};

}  // namespace fc
