// double instantiations of the particle pass (pass.cuh).
#include "pass.cuh"

namespace galpic {

int launch_pass_fp64(pic_sim* s, int mode, cudaStream_t st) {
    return mode == PASS_STEP ? pass_margin<double, PASS_STEP>(s, st) : pass_margin<double, PASS_DEPOSIT>(s, st);
}

}  // namespace galpic
