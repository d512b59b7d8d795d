// Variants for TESS 2-min style windows (W up to 768).
#include "umi_variants.h"
UMI_DEFINE_VARIANT(8, 46)
UMI_DEFINE_VARIANT(16, 48)
