// refine.cu -- two-level grid refinement of Sec. 4 (placeholder until built).
#include "lb_runtime.h"

lb_status refine_setup(lb_ctx *ctx, const lb_config *, const float *) {
    return lbrt::fail(ctx, LB_EINVAL, "grid refinement is not available in this build");
}
void refine_destroy(lb_ctx *) {}
bool refine_contains(const lb_ctx *, int, int) { return false; }
lb_status refine_set_receivers(lb_ctx *, const int *, int) { return LB_OK; }
lb_status refine_after_set_state(lb_ctx *) { return LB_OK; }
lb_status refine_step(lb_ctx *ctx, int) { return lbrt::fail(ctx, LB_ESTATE, "no patch"); }
lb_status refine_overlay_pressure(lb_ctx *, float *) { return LB_OK; }
