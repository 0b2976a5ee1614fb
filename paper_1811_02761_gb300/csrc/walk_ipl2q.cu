// walk_ipl2q.cu -- instances of the tree walk with up to 2 i-particles per lane,
// nodes with quadrupoles (separate translation unit so the instances compile
// in parallel).
#include "walk_impl.cuh"

namespace nb {
template cudaError_t launch_walk_ipl<2, true>(cudaStream_t, const WalkArgs &, const WalkShape &, int);
}  // namespace nb
