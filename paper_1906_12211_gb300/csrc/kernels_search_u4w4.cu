// Instantiations of the search kernel with 4 positions per lane per streaming
// step and 4 warps per query (one per padded dimension class).
#include "search_kernel.cuh"

namespace pf {
namespace skern {

Kernel pick_u4w4(int d_pad) { return pick_nt<4, 4, false>(d_pad); }

}  // namespace skern
}  // namespace pf
