// The k > 63 instances of the kernels (four-word k-mers, reference slots):
// the same source as twopaco_kernels.cu, compiled as a second translation
// unit so that the two build in parallel.
#define TWOPACO_WIDE_ONLY 1
#include "twopaco_kernels.cu"
