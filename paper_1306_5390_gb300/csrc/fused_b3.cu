// Fused kernel instances for beta = 3 .. 7.
#include "fused.cuh"

namespace hg {
extern const FusedEntry kFusedB3[] = {
    fused_entry<3, 1>(), fused_entry<3, 2>(), fused_entry<4, 1>(), fused_entry<4, 2>(),
    fused_entry<5, 1>(), fused_entry<6, 1>(), fused_entry<7, 1>(),
};
extern const int kFusedB3Count = sizeof(kFusedB3) / sizeof(kFusedB3[0]);
}  // namespace hg
