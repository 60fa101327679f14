// NCL outer loop and interior-point inner loop (placeholder until the
// device-resident control is wired in).
#include "handle.h"

namespace scopf {
int ncl_solve_impl(scopf_handle *h, const scopf_state *warm, scopf_result *res) {
    (void)h; (void)warm; (void)res;
    return SCOPF_ERR_INVALID_ARG;
}
}  // namespace scopf
