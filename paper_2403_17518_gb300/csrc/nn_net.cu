// Deblurring network state (Section 2.4): owned by the context.
#include "nn_api.h"

namespace dhfwi {

struct NetState {
    int placeholder = 0;
};

void net_destroy(NetState *net) { delete net; }

}  // namespace dhfwi
