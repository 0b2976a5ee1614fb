// walk_ipl4.cu -- instances of the tree walk with up to 4 i-particles per lane,
// monopole nodes (separate translation unit so the instances compile in parallel).
#include "walk_impl.cuh"

namespace nb {
template cudaError_t launch_walk_ipl<4, false>(cudaStream_t, const WalkArgs &, const WalkShape &, int);
}  // namespace nb
