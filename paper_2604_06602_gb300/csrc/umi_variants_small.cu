// Variants for short windows (W <= 192): one to eight lanes per window.
#include "umi_variants.h"
UMI_DEFINE_VARIANT(1, 8)
UMI_DEFINE_VARIANT(1, 16)
UMI_DEFINE_VARIANT(1, 32)
UMI_DEFINE_VARIANT(2, 32)
UMI_DEFINE_VARIANT(4, 32)
UMI_DEFINE_VARIANT(8, 24)
