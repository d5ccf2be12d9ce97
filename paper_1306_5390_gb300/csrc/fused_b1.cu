// Fused kernel instances for beta = 1.
#include "fused.cuh"

namespace hg {
extern const FusedEntry kFusedB1[] = {
    fused_entry<1, 1>(), fused_entry<1, 2>(), fused_entry<1, 3>(),
    fused_entry<1, 4>(), fused_entry<1, 6>(), fused_entry<1, 8>(), fused_entry<1, 8, 128>(),
};
extern const int kFusedB1Count = sizeof(kFusedB1) / sizeof(kFusedB1[0]);
}  // namespace hg
