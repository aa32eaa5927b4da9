// The preconditioner's fused column pass in its 512- and 1024-thread shapes
// (columns of 2048 or 4096 complex values at ratios 2 and 4), built as a
// translation unit of its own so that it compiles beside precond.cu.
#define PS_PREC_WIDE
#include "precond.cu"
