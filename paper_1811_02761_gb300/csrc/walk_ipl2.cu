// walk_ipl2.cu -- instances of the tree walk with up to 2 i-particles per lane,
// monopole nodes (separate translation unit so the instances compile in parallel).
#include "walk_impl.cuh"

namespace nb {
template cudaError_t launch_walk_ipl<2, false>(cudaStream_t, const WalkArgs &, const WalkShape &, int);
}  // namespace nb
