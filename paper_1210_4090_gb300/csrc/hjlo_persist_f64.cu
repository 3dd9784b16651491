// hjlo_persist_f64.cu -- the persistent batched pass, binary64 storage.
#define HJLO_KT double
#define HJLO_KNAME f64
#include "hjlo_persist.inc"
