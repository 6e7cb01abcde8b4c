/* A plain C99 caller of the library: includes the public header as C, links
 * liblpf.so and calls the entry points that need no GPU (defaults, the device
 * footprint of a stream, argument errors, error names).  Prints one line of
 * results; the test compares them with the same calls made through ctypes. */
#include <stdio.h>
#include <string.h>

#include "lpf.h"

int main(void) {
    lpf_params p;
    lpf_default_params(&p);
    double freqs[16];
    for (int i = 0; i < 16; ++i) freqs[i] = (i < 8 ? 57.6 : 61.2) + ((i % 8) + 0.5) * 0.1953125;
    double dms[251];
    for (int d = 0; d < 251; ++d) dms[d] = (double)d;
    size_t bytes = 0;
    int rc = lpf_stream_footprint(1024, 1024, 16, freqs, 251, dms, 48, &p, &bytes);
    size_t bytes_null = 0;
    int rc_null = lpf_stream_footprint(1024, 1024, 16, freqs, 251, dms, 48, NULL, &bytes_null);
    size_t unused = 0;
    int rc_depth = lpf_stream_footprint(1024, 1024, 16, freqs, 251, dms, 47, &p, &unused);
    lpf_params bad = p;
    bad.box_r = 17;
    int rc_arg = lpf_stream_footprint(1024, 1024, 16, freqs, 251, dms, 48, &bad, &unused);
    lpf_params sup = p;
    sup.suppress_steady = 8;
    size_t bytes_sup = 0;
    int rc_sup = lpf_stream_footprint(1024, 1024, 16, freqs, 251, dms, 48, &sup, &bytes_sup);
    const char* name = lpf_strerror(LPF_E_DEPTH);
    printf("%d %zu %d %zu %d %d %d %d %.1f %s %d %zu %zu\n", rc, bytes, rc_null, bytes_null, rc_depth, rc_arg,
           p.box_r, p.cand_cap, (double)p.kappa, strlen(name) > 0 ? "named" : "unnamed", rc_sup, bytes_sup,
           sizeof(lpf_params));
    return 0;
}
