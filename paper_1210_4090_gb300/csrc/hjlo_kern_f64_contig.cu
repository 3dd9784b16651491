// Axis-pass kernels for binary64 storage, lines along the contiguous axis.
#define HJLO_KT double
#define HJLO_KL LAYOUT_CONTIG
#define HJLO_KNAME f64_contig
#include "hjlo_kern.inc"
