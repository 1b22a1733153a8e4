// Internal interface between the C ABI host code (api.cu) and the deblurring
// network (nn_*.cu).  Not part of the C ABI.
#pragma once

struct dhfwi_ctx;

namespace dhfwi {

struct NetState;

void net_destroy(NetState *net);

// Context accessors implemented in api.cu.
NetState *&ctx_net(dhfwi_ctx *ctx);
int ctx_device(dhfwi_ctx *ctx);
void ctx_set_error(dhfwi_ctx *ctx, const char *msg);
void ctx_begin(dhfwi_ctx *ctx);
void ctx_count_launches(dhfwi_ctx *ctx, long long n);

}  // namespace dhfwi
