// Host exports of the device geometry and Philox functions (no device work).
#include "../../include/mctrg.h"
#include "../../include/mctrg_host.h"
#include "common.cuh"

extern "C" int mctrg_plan_level(int L, int k, uint8_t* parity, int64_t* parents) {
  if (L < 2 || L > 4096 || (L & (L - 1))) return MCTRG_EINVAL;
  int m = 0;
  while ((1 << m) < L) ++m;
  if (k < 0 || k >= 2 * m) return MCTRG_EINVAL;
  const int64_t N = mctrg::level_count(L, k);
  if (parity)
    for (int64_t t = 0; t < N; ++t) parity[t] = (uint8_t)mctrg::tensor_parity(L, k, t);
  if (parents)
    for (int64_t c = 0; c < N / 2; ++c) mctrg::tensor_parents(L, k, c, parents + 4 * c);
  return MCTRG_OK;
}

extern "C" double mctrg_philox_uniform(uint64_t seed, uint32_t traj, uint32_t level, uint32_t tensor,
                                       uint32_t t) {
  return mctrg::philox_uniform(seed, traj, level, tensor, t);
}
