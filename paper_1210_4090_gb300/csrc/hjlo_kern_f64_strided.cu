// Axis-pass kernels for binary64 storage, lines along the a strided axis.
#define HJLO_KT double
#define HJLO_KL LAYOUT_STRIDED
#define HJLO_KNAME f64_strided
#include "hjlo_kern.inc"
