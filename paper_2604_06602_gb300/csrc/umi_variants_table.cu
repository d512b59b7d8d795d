// The compiled variant table (kernels are defined in umi_variants_*.cu).
#include "umi_variants.h"

UMI_VARIANT_LIST(UMI_DECLARE_VARIANT)

namespace umi {

namespace {
struct Table {
    Variant v[64];
    int n = 0;
    Table()
    {
#define UMI_TABLE_ENTRY(G_, R_, M_) UMI_VNAME(fill_, G_, R_, M_)(&v[n++]);
        UMI_VARIANT_LIST(UMI_TABLE_ENTRY)
#undef UMI_TABLE_ENTRY
    }
};
}  // namespace

const Variant *variant_table(int *count)
{
    static const Table table;
    if (count) *count = table.n;
    return table.v;
}

}  // namespace umi
