// emul.cu -- emulated-precision paths (filled in by the Ozaki / TF32 kernels).
#include "emul.cuh"

namespace dbcsr {

int dgemm_emulated(int64_t, int64_t, int64_t, double, const double*, int64_t, const double*, int64_t, double,
                   double*, int64_t, const dbcsr_opts&) {
    return fail(DBCSR_ERR_ARG, "emulated precision is not available in this build");
}

int smm_emulated(const SmmArgs&, int, int, int, const dbcsr_opts&) {
    return fail(DBCSR_ERR_ARG, "emulated precision is not available in this build");
}

}  // namespace dbcsr
