// Instantiations of the search kernel with 8 positions per lane per streaming
// step and 8 warps per query (one per padded dimension class).
#include "search_kernel.cuh"

namespace pf {
namespace skern {

Kernel pick_u8w8(int d_pad) { return pick_nt<8, 8, false>(d_pad); }

}  // namespace skern
}  // namespace pf
