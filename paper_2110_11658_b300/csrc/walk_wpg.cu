// Walk variants with several warps per group (threads per group 64 and 128): the
// group's first warp walks the tree, every warp evaluates the queues for its own
// 32 targets (walk_kernel.cuh).  A translation unit of its own so that the two
// halves of the walk's instantiations compile in parallel.
#include "walk_kernel.cuh"

namespace p3t {

template int dispatch_walk_wpg<2>(p3t_ctx *, const WalkArgs &, bool, int, bool, bool, bool);
template int dispatch_walk_wpg<4>(p3t_ctx *, const WalkArgs &, bool, int, bool, bool, bool);

}  // namespace p3t
