// hjlo_persist_f32.cu -- the persistent batched pass, binary32 storage.
#define HJLO_KT float
#define HJLO_KNAME f32
#include "hjlo_persist.inc"
