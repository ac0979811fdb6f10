// Tensor-core (tcgen05) convolutions: placeholder until the BF16 / FP8 kernels land.
#include "lnr_internal.h"

namespace lnr {

bool tc_available() { return false; }

cudaError_t tc_prepare_layer(ConvLayer&, lnr_precision) { return cudaErrorNotSupported; }

void tc_conv(const ConvLayer&, lnr_precision, const void*, const void*, void*, void*, const float*,
             const float*, float*, int, int, int, cudaStream_t) {}

}  // namespace lnr
