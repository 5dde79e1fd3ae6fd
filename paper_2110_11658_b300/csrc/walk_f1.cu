// The mixed walks with one warp per group, cell form 1 (the r^-5 quadrupole term; walk_kernel.cuh), in a
// translation unit of their own so that the walk's instantiations compile in parallel.
#include "walk_kernel.cuh"

namespace p3t {

template int mixed_walk<1>(p3t_ctx *, const WalkArgs &, int, int, bool, bool, bool);

}  // namespace p3t
