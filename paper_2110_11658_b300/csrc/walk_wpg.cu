// Walk variants with several warps per group (threads per group 64 and 128): the
// group's first warp walks the tree, every warp evaluates the queues for its own
// 32 targets (walk_kernel.cuh).  Translation units of their own (cell form 1 here,
// the FP64 form and cell form 2 in walk_wpg2.cu) so that the walk's instantiations
// compile in parallel.
#include "walk_kernel.cuh"

namespace p3t {

#define P3T_WPG(W, F) template int dispatch_walk_wpg<W, F>(p3t_ctx *, const WalkArgs &, int, bool, bool, bool);
P3T_WPG(2, 1)
P3T_WPG(4, 1)
#undef P3T_WPG

}  // namespace p3t
