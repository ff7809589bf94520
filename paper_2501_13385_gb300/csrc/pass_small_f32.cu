// FP32 sampled pass for rank bucket 8: kernels per register size RC = 5..8
// (the problem's largest TT-rank) and mode class, single-problem and batched;
// RC = 1..4 (bucket 4) live in pass_small_f32_r4.cu.
#include "omega_pass.cuh"

int ttc_pass_small_f32(int RC, const PassLaunch& L) {
  using namespace ttc_pass;
  switch (RC) {
    case 5: return launch<float, 8, 5>(L);
    case 6: return launch<float, 8, 6>(L);
    case 7: return launch<float, 8, 7>(L);
    case 8: return launch<float, 8, 8>(L);
    default: return ttc_pass_small_f32_r4(RC, L);
  }
}
