// FP64 sampled pass for rank buckets 4 and 8: one kernel per register size
// RC = 1..8 (the problem's largest TT-rank), single-problem and batched.
#include "omega_pass.cuh"

int ttc_pass_small_f64(int RC, const PassLaunch& L) {
  using namespace ttc_pass;
  switch (RC) {
    case 1: return launch<double, 4, 1>(L);
    case 2: return launch<double, 4, 2>(L);
    case 3: return launch<double, 4, 3>(L);
    case 4: return launch<double, 4, 4>(L);
    case 5: return launch<double, 8, 5>(L);
    case 6: return launch<double, 8, 6>(L);
    case 7: return launch<double, 8, 7>(L);
    case 8: return launch<double, 8, 8>(L);
    default: return TTC_EUNSUPPORTED;
  }
}
