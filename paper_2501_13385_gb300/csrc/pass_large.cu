// Sampled pass for rank buckets 16 and 32 (FP32 and FP64): one block per
// chunk, register arrays of the bucket size.
#include "omega_pass.cuh"

int ttc_pass_large(bool f32, int R, const PassLaunch& L) {
  using namespace ttc_pass;
  if (R == 16) return f32 ? launch<float, 16, 16>(L) : launch<double, 16, 16>(L);
  return f32 ? launch<float, 32, 32>(L) : launch<double, 32, 32>(L);
}

// kernels whose shared memory exceeds the default 48 KiB (outside any capture)
int ttc_pass_opt_in_large() {
  using namespace ttc_pass;
  TTC_TRY((opt_in<float, 16, 16>()));
  TTC_TRY((opt_in<float, 32, 32>()));
  TTC_TRY((opt_in<double, 16, 16>()));
  TTC_TRY((opt_in<double, 32, 32>()));
  return TTC_OK;
}
