// Mixed-precision operator application (tcgen05 tensor-core DST); built in
// a following step.
#include "internal.h"

namespace kfbi {

struct TcDst {
  long long bytes = 0;
};

TcDst* tc_create(kfbi_domain*) {
  throw Status{KFBI_ERR_UNSUPPORTED, "KFBI_MIXED_TF32 is not built yet"};
}
void tc_destroy(TcDst* tc) { delete tc; }
void tc_apply(kfbi_domain*, double, double, const double*, int, const double*, double*, int, bool,
              cudaStream_t) {
  throw Status{KFBI_ERR_UNSUPPORTED, "KFBI_MIXED_TF32 is not built yet"};
}
long long tc_bytes(const TcDst* tc) { return tc ? tc->bytes : 0; }

}  // namespace kfbi
