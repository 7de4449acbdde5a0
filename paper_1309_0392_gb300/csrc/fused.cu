// Fused path (dyadic tiles): not built yet.
#include "gbh_internal.h"

namespace gbh {

bool fused_supported(const Geom &, int, int) { return false; }

int fused_transform(void *, const Geom &, int, int, const gbh_options *, cudaStream_t)
{
    return GBH_EUNSUPPORTED;
}

}  // namespace gbh
