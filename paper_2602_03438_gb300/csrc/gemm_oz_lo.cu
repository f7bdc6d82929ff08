// The sliced BF16 complex product with 5 digits per value: 15 slice pairs instead of
// 36, error ~2^-34 of the row x column norms of its operands.  It serves products whose
// result is a small correction, such as X (I - M X) in the refinement of an inverse,
// where I - M X is below ~1e-3 and the correction needs only that relative accuracy.
// The kernels are those of gemm_oz.cu, compiled here a second time.
#define NEGF_OZ_DIGITS 5
#define NEGF_OZ_LOW 1
#include "gemm_oz.cu"
