// hope_stage_d_lo.cu -- instantiations of the stage sequences for double, orders 3, 5, 7.
#include "hope_stage.cuh"

namespace hope {

stage_fn stage_entry_d_lo(int k) {
  switch (k) {
    case 3: return stage_all<double, 3>;
    case 5: return stage_all<double, 5>;
    case 7: return stage_all<double, 7>;
  }
  return nullptr;
}

vjp_fn vjp_entry_d_lo(int k) {
  switch (k) {
    case 3: return stage_vjp_all<double, 3>;
    case 5: return stage_vjp_all<double, 5>;
    case 7: return stage_vjp_all<double, 7>;
  }
  return nullptr;
}

int smem_attr_entry_d_lo(int k) {
  switch (k) {
    case 3: return set_smem_attr<double, 3>();
    case 5: return set_smem_attr<double, 5>();
    case 7: return set_smem_attr<double, 7>();
  }
  return -1;
}

}  // namespace hope
