// The mixed walks with one warp per group, cell form 2 (the r^-3 quadrupole term; walk_kernel.cuh), in a
// translation unit of their own so that the walk's instantiations compile in parallel.
#include "walk_kernel.cuh"

namespace p3t {

template int mixed_walk<2>(p3t_ctx *, const WalkArgs &, int, int, bool, bool, bool);

}  // namespace p3t
