// Random initial MPS (block2 paper, Sec. 2.1.6 "Initial guesses" (i) and (ii)).
#include "algo.hpp"

b2_mps_s* b2_mps_random_impl(b2::Ctx* ctx, b2_mpo_s* mpo, int M, const double* occ,
                             uint64_t seed) {
  (void)ctx; (void)mpo; (void)M; (void)occ; (void)seed;
  throw b2::Error(B2_EUNSUPPORTED, "b2_mps_random is not implemented yet");
}
