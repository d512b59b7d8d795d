// Variants for long windows (W up to 4096): a full warp per window.
#include "umi_variants.h"
UMI_DEFINE_VARIANT(32, 48)
UMI_DEFINE_VARIANT(32, 68)
UMI_DEFINE_VARIANT(32, 128)
