/* A plain C99 program against include/mk.h and libmk.so: the boundary is
   a C ABI, usable without Python or torch.  It calls host-only entry points
   (no GPU needed) and prints one "name value" line per check for
   tests/test_host_library.py to compare. */
#include <stdio.h>
#include <string.h>

#include "mk.h"

int main(void) {
    mk_program p;
    int32_t pos = -1;
    mk_cert c;
    mk_census_cfg cfg;
    int rc;

    printf("version %d\n", mk_version());

    rc = mk_compile("[]p -> p", &p, &pos);
    printf("compile %d nvars %d nodes %d\n", rc, (int)p.nvars, (int)p.nodes);
    rc = mk_compile("[]p ->", &p, &pos);
    printf("syntax %d %s\n", rc, rc == MK_E_SYNTAX ? "ok" : "bad");
    printf("strerror %s\n", mk_strerror(MK_E_SYNTAX) ? "set" : "null");

    /* Prop. 5: successor masks (2,4,8,16,32,0), alpha_3 false and alpha_2
       true at world 0 */
    memset(&c, 0, sizeof(c));
    c.phi = "[]<>[]<>T";
    c.psi = "[]<>[]<>[]<>T";
    c.n = 6;
    c.cls = 0;
    c.world = 0;
    c.succ[0] = 2; c.succ[1] = 4; c.succ[2] = 8; c.succ[3] = 16; c.succ[4] = 32; c.succ[5] = 0;
    printf("certify %d\n", mk_certify(&c));
    c.world = 5;   /* the dead end: both formulas hold there */
    printf("certify_dead_end %d\n", mk_certify(&c));

    printf("s4_5 %llu\n", (unsigned long long)mk_class_frames(MK_CLASS_S4, 5));
    printf("s5_5 %llu\n", (unsigned long long)mk_class_frames(MK_CLASS_S5, 5));

    memset(&cfg, 0, sizeof(cfg));
    cfg.classes = MK_CLASS_K | MK_CLASS_S4;
    cfg.n_min = 1;
    cfg.n_max = 5;
    cfg.frame_hi = ~(uint64_t)0;
    printf("workspace %s\n", mk_census_workspace_size(&cfg, 64) > 0 ? "positive" : "zero");
    cfg.n_max = 9;   /* beyond the exhaustive limit */
    printf("workspace_bad %llu\n", (unsigned long long)mk_census_workspace_size(&cfg, 64));
    return 0;
}
