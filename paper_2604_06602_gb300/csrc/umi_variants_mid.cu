// Variants for TESS 2-min style windows (W up to 384): the autotuner picks
// among lane-group widths 8, 16 and 32.
#include "umi_variants.h"
UMI_DEFINE_VARIANT(8, 46, 2)
UMI_DEFINE_VARIANT(8, 46, 3)
UMI_DEFINE_VARIANT(16, 24, 4)
UMI_DEFINE_VARIANT(32, 12, 4)
