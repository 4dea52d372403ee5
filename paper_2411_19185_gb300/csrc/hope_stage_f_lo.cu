// hope_stage_f_lo.cu -- instantiations of the stage sequences for float, orders 3, 5, 7.
#include "hope_stage.cuh"

namespace hope {

stage_fn stage_entry_f_lo(int k) {
  switch (k) {
    case 3: return stage_all<float, 3>;
    case 5: return stage_all<float, 5>;
    case 7: return stage_all<float, 7>;
  }
  return nullptr;
}

vjp_fn vjp_entry_f_lo(int k) {
  switch (k) {
    case 3: return stage_vjp_all<float, 3>;
    case 5: return stage_vjp_all<float, 5>;
    case 7: return stage_vjp_all<float, 7>;
  }
  return nullptr;
}

int smem_attr_entry_f_lo(int k) {
  switch (k) {
    case 3: return set_smem_attr<float, 3>();
    case 5: return set_smem_attr<float, 5>();
    case 7: return set_smem_attr<float, 7>();
  }
  return -1;
}

}  // namespace hope
