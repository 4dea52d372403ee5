// hope_stage_d_hi.cu -- instantiations of the stage sequences for double, orders 9, 11.
#include "hope_stage.cuh"

namespace hope {

stage_fn stage_entry_d_hi(int k) {
  switch (k) {
    case 9: return stage_all<double, 9>;
    case 11: return stage_all<double, 11>;
  }
  return nullptr;
}

vjp_fn vjp_entry_d_hi(int k) {
  switch (k) {
    case 9: return stage_vjp_all<double, 9>;
    case 11: return stage_vjp_all<double, 11>;
  }
  return nullptr;
}

int smem_attr_entry_d_hi(int k) {
  switch (k) {
    case 9: return set_smem_attr<double, 9>();
    case 11: return set_smem_attr<double, 11>();
  }
  return -1;
}

}  // namespace hope
