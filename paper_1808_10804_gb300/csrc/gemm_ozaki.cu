// Mixed-precision (Ozaki-split BF16 on tcgen05) grouped GEMM -- placeholder
// until the tensor-core kernel lands.
#include "bst_internal.h"

namespace bst {

struct OzakiPlan {};

void ozaki_prepare(Ctx*, ContractPlan*) { throw Error(BST_E_UNSUPPORTED, "BST_OZAKI not built yet"); }
void run_gemm_ozaki(Ctx*, ContractPlan*, const double*, const double*, double*, cudaStream_t) {
  throw Error(BST_E_UNSUPPORTED, "BST_OZAKI not built yet");
}
void ozaki_free(OzakiPlan* oz) { delete oz; }
void run_gemm_ozaki_probs(Ctx*, const std::string&, const std::vector<GemmProb>&, const double*, const double*,
                          double*, cudaStream_t) {
  throw Error(BST_E_UNSUPPORTED, "BST_OZAKI not built yet");
}

}  // namespace bst
