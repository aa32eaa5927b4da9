// The CG-loop site kernels of cg_fast.cu for ratio 4 and kernel radii 12, 14
// and 16 (the paper's 29 x 29 support is R = 14), built as a translation unit
// of their own.
#define PS_SITE_WIDE
#include "cg_fast.cu"
