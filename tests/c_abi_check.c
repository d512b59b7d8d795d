/* Compiled by tests/test_abi.py with a C99 compiler: include/umi.h must be
 * valid C, and the host-only calls must work through the shared library
 * without any GPU work. */
#include <stdio.h>
#include <string.h>

#include "umi.h"

int main(void)
{
    umi_params p;
    umi_default_params(&p);
    if (p.alpha != 2.0f || p.c != 5.0f || p.iters != 5 || p.min_valid != -1 ||
        p.scale_mode != UMI_SCALE_UPPER_RMS)
        return 1;
    if (umi_window_length(2.0 / 1440.0, 0.5) != 361) return 2;
    if (umi_window_length(29.4 / 1440.0, 0.5) != 25) return 3;
    if (umi_window_length(0.0, 0.5) != -1) return 4;
    /* Validation happens on the host: an even window is rejected before any
     * device work, with a message. */
    if (umi_detrend(NULL, 10, 4, &p, NULL, NULL, NULL) != UMI_ERR_INVALID_ARG) return 5;
    if (strlen(umi_last_error()) == 0) return 6;
    umi_segment_params sp;
    umi_default_segment_params(&sp);
    if (sp.gap_min != 0 || sp.min_seg != -1) return 7;
    umi_server_config cfg;
    umi_server_default_config(&cfg);
    if (cfg.mem_budget_bytes != (40ull << 30)) return 8;
    printf("%s\n", umi_version());
    return 0;
}
