// hope_stage_f_hi.cu -- instantiations of the stage sequences for float, orders 9, 11.
#include "hope_stage.cuh"

namespace hope {

stage_fn stage_entry_f_hi(int k) {
  switch (k) {
    case 9: return stage_all<float, 9>;
    case 11: return stage_all<float, 11>;
  }
  return nullptr;
}

vjp_fn vjp_entry_f_hi(int k) {
  switch (k) {
    case 9: return stage_vjp_all<float, 9>;
    case 11: return stage_vjp_all<float, 11>;
  }
  return nullptr;
}

int smem_attr_entry_f_hi(int k) {
  switch (k) {
    case 9: return set_smem_attr<float, 9>();
    case 11: return set_smem_attr<float, 11>();
  }
  return -1;
}

}  // namespace hope
