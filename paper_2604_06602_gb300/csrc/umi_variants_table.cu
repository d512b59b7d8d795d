// The compiled variant table (launchers are defined in umi_variants_*.cu).
#include "umi_variants.h"

UMI_VARIANT_LIST(UMI_DECLARE_VARIANT)

namespace umi {

const Variant *variant_table(int *count)
{
#define UMI_TABLE_ENTRY(G_, R_, M_)                                                       \
    {G_, R_, M_, UMI_VNAME(launch_v, G_, R_, M_), UMI_VNAME(launch_d, G_, R_, M_),         \
     UMI_VNAME(kernel_v, G_, R_, M_)(), UMI_VNAME(kernel_d, G_, R_, M_)()},
    static const Variant table[] = {UMI_VARIANT_LIST(UMI_TABLE_ENTRY)};
#undef UMI_TABLE_ENTRY
    if (count) *count = (int)(sizeof(table) / sizeof(table[0]));
    return table;
}

}  // namespace umi
