/*
 * mctrg_host.h - host-only helpers of the MC-TRG library (no device work).
 *
 * Exposes the TRG geometry the device kernels compute on the fly, so that it
 * can be checked without a GPU.  Levin-Nave coarse-graining (Sec. III) on an
 * L x L torus: level k has L^2 / 2^k tensors; each level-(k+1) tensor is the
 * plaquette whose top-left corner p is a sublattice-A tensor of level k, and
 * its four parents are p, p+a1, p+a2 and p+a1+a2 (contributing the halves
 * F3, F4, F2 and F1).  Numbering: level 0 tensor (x, y) has id y L + x;
 * level k+1 tensors are numbered by the level-k id of their top-left parent.
 */
#ifndef MCTRG_HOST_H
#define MCTRG_HOST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Geometry of level k (0 <= k < 2 log2 L) of an L x L torus, L a power of two
 * with 2 <= L <= 4096.  parity (host, L^2/2^k bytes, may be NULL) receives 0
 * for sublattice A and 1 for B.  parents (host, 4 * L^2/2^(k+1) int64, may be
 * NULL) receives, for each tensor c of level k+1, the level-k ids of
 * (p, p+a1, p+a2, p+a1+a2).  Returns MCTRG_OK or MCTRG_EINVAL. */
int mctrg_plan_level(int L, int k, uint8_t* parity, int64_t* parents);

/* Philox4x32-10 uniform of draw step t for (seed, trajectory, level, tensor),
 * the exact value the device sampler consumes. */
double mctrg_philox_uniform(uint64_t seed, uint32_t traj, uint32_t level, uint32_t tensor,
                            uint32_t t);

#ifdef __cplusplus
}
#endif
#endif /* MCTRG_HOST_H */
