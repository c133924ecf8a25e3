// Tensor-core (tcgen05 / TMEM) kernels of the mixed-precision path.
#include "common.cuh"

namespace dpg {

bool tc_available(const Model*) { return false; }

dp_status launch_tc_setup(Model* m) {
  m->last_error = "tensor-core path not built";
  return DP_ERR_UNSUPPORTED;
}

}  // namespace dpg
