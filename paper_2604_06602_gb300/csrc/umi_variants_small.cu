// Variants for short windows (W <= 192): one to eight lanes per window.
#include "umi_variants.h"
UMI_DEFINE_VARIANT(1, 8, 4)
UMI_DEFINE_VARIANT(1, 16, 4)
UMI_DEFINE_VARIANT(1, 26, 4)
UMI_DEFINE_VARIANT(1, 32, 3)
UMI_DEFINE_VARIANT(2, 32, 3)
UMI_DEFINE_VARIANT(4, 32, 3)
UMI_DEFINE_VARIANT(8, 24, 3)
