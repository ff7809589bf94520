// Sampled pass for rank buckets 16 and 32 (FP32 and FP64): warp-per-chunk
// kernels for the first and last modes, block-per-chunk kernels for the
// interior modes, register arrays of RC = 16 (bucket 16), 24 or 32 (bucket 32).
#include "omega_pass.cuh"

int ttc_pass_large(bool f32, int R, int RC, const PassLaunch& L) {
  using namespace ttc_pass;
  if (R == 16) return f32 ? launch<float, 16, 16>(L) : launch<double, 16, 16>(L);
  if (RC <= 24) return f32 ? launch<float, 32, 24>(L) : launch<double, 32, 24>(L);
  return f32 ? launch<float, 32, 32>(L) : launch<double, 32, 32>(L);
}

// kernels whose shared memory exceeds the default 48 KiB (outside any capture)
int ttc_pass_opt_in_large() {
  using namespace ttc_pass;
  TTC_TRY((opt_in<float, 16, 16>()));
  TTC_TRY((opt_in<float, 32, 24>()));
  TTC_TRY((opt_in<float, 32, 32>()));
  TTC_TRY((opt_in<double, 16, 16>()));
  TTC_TRY((opt_in<double, 32, 24>()));
  TTC_TRY((opt_in<double, 32, 32>()));
  return TTC_OK;
}
