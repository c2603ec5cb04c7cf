// k_mg2d_alt2.cu -- the coarse-level V-cycle tile shapes that the autotuner can choose instead of
// the default (TMA staging only), compiled apart from k_mg2d.cu so that the units build in parallel.
#include "k_mg2d_impl.cuh"

namespace plsqr {

PLSQR_MG2D_ALT_COARSE()

}  // namespace plsqr
