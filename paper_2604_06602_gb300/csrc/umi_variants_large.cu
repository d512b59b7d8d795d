// Variants for long windows (W up to 4096).
#include "umi_variants.h"
UMI_DEFINE_VARIANT(16, 48, 2)
UMI_DEFINE_VARIANT(32, 48, 2)
UMI_DEFINE_VARIANT(32, 68, 2)
UMI_DEFINE_VARIANT(32, 128, 1)
