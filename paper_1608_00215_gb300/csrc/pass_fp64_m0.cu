// double particle-pass kernels at tile margin 0 (pass.cuh).
#include "pass.cuh"

namespace galpic {

int pass_fp64_margin0(pic_sim* s, int mode, cudaStream_t st, const void* descs, int nruns) {
    const ManyLaunch m{descs, nruns};
    const ManyLaunch* many = descs ? &m : nullptr;
    return mode == PASS_STEP ? pass_order<double, PASS_STEP, 0>(s, st, many)
                             : pass_order<double, PASS_DEPOSIT, 0>(s, st, nullptr);
}

}  // namespace galpic
