// Instantiations of the search kernel with 8 positions per lane per streaming
// step and 4 warps per query that can stream a round
// flat (launch shapes with flat_fill > 0; one per padded dimension class).
#include "search_kernel.cuh"

namespace pf {
namespace skern {

Kernel pick_u8w4_flat(int d_pad) { return pick_nt<8, 4, true>(d_pad); }

}  // namespace skern
}  // namespace pf
