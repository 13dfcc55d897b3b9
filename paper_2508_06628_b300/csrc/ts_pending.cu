// ts_pending.cu -- entry points still to be written return TS_ERR_UNSUPPORTED.
#include "ts_api.h"
using namespace ts;
extern "C" ts_status ts_batch_compact_admit(ts_batch* b, const ts_state*, const uint8_t*, const ts_host_systems*,
                                            ts_state*, const ts_fire_state*, const double*, ts_fire_state*, double*,
                                            const ts_fire_params*, void*) {
  return fail(b, TS_ERR_UNSUPPORTED, "not built");
}
extern "C" ts_status ts_autotune(ts_batch* b, ts_state*, void*) { return fail(b, TS_ERR_UNSUPPORTED, "not built"); }
namespace ts { void autotune_load(ts_batch*) {} }
