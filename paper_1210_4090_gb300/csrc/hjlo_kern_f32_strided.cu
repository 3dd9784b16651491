// Axis-pass kernels for binary32 storage, lines along the a strided axis.
#define HJLO_KT float
#define HJLO_KL LAYOUT_STRIDED
#define HJLO_KNAME f32_strided
#include "hjlo_kern.inc"
