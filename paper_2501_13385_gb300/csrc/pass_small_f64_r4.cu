// FP64 sampled pass for rank bucket 4: kernels per register size RC = 1..4
// and mode class, single-problem and batched.
#include "omega_pass.cuh"

int ttc_pass_small_f64_r4(int RC, const PassLaunch& L) {
  using namespace ttc_pass;
  switch (RC) {
    case 1: return launch<double, 4, 1>(L);
    case 2: return launch<double, 4, 2>(L);
    case 3: return launch<double, 4, 3>(L);
    case 4: return launch<double, 4, 4>(L);
    default: return TTC_EUNSUPPORTED;
  }
}
