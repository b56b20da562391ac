#include "sigma_tc.cuh"

namespace kpm {

void TcSigma::init(const SpinTables&, const SpinTables&, const double*, const double*, int,
                   cudaStream_t) {
    KPM_THROW(KPM_EUNSUPPORTED, "KPM_MIXED is not available in this build");
}

void TcSigma::apply(const float*, float*, int, cudaStream_t) {
    KPM_THROW(KPM_EUNSUPPORTED, "KPM_MIXED is not available in this build");
}

}  // namespace kpm
