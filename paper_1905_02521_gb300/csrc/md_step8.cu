// md_step8.cu -- the cooperative step kernel with 8 lanes per bead-atom
// (instantiated in a translation unit of its own so that the variants compile in
// parallel).
#include "md_kernels.cuh"

namespace qtb {

cudaError_t step_prepare_l8(MdLaunch &m, int stage_entries) { return step_prepare_lanes<8>(m, stage_entries); }

cudaError_t step_force_l8(const Dev &d, const MdLaunch &m, const PairTabT<float> &Tf, const PairTabT<double> &Td,
                          int kick, int j, int cur, int adv, int rec, cudaStream_t st)
{
    return step_force_lanes<8>(d, m, Tf, Td, kick, j, cur, adv, rec, st);
}

}  // namespace qtb
