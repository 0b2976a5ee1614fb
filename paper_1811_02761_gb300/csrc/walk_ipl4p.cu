// walk_ipl4p.cu -- instances of the warp-specialised tree walk with up to 4
// i-particles per lane (separate translation unit so the instances compile
// in parallel).
#include "walk_pipe.cuh"

namespace nb {
template cudaError_t launch_walk_pipe_ipl<4>(cudaStream_t, const WalkArgs &, const WalkShape &, int);
}  // namespace nb
