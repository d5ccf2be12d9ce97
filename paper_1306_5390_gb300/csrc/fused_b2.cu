// Fused kernel instances for beta = 2.
#include "fused.cuh"

namespace hg {
extern const FusedEntry kFusedB2[] = {
    fused_entry<2, 1>(), fused_entry<2, 2>(), fused_entry<2, 3>(), fused_entry<2, 4>(), fused_entry<2, 4, 128>(),
};
extern const int kFusedB2Count = sizeof(kFusedB2) / sizeof(kFusedB2[0]);
}  // namespace hg
