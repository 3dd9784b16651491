// Axis-pass kernels for binary32 storage, lines along the contiguous axis.
#define HJLO_KT float
#define HJLO_KL LAYOUT_CONTIG
#define HJLO_KNAME f32_contig
#include "hjlo_kern.inc"
