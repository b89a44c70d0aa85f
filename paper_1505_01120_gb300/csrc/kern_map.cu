// kern_map.cu -- MapCL (materialised output) kernels and the keyed fold pass.
#include "kernels.cuh"

namespace scl {

namespace {
constexpr int kMapBlock = 256;
constexpr int kMapIpt = 4;
}  // namespace

const void* fold_kernel_fn() { return (const void*)&dev::k_keyed_fold<kFoldBlock>; }

int map_kernel_block() { return kMapBlock; }
int map_kernel_ipt() { return kMapIpt; }

const void* map_kernel_fn(int kind, int aligned) {
    switch (kind) {
        case K_U32_IDENT:
            return aligned ? (const void*)&dev::k_map<kMapBlock, kMapIpt, K_U32_IDENT, true>
                           : (const void*)&dev::k_map<kMapBlock, kMapIpt, K_U32_IDENT, false>;
        case K_U32_MIX32:
            return aligned ? (const void*)&dev::k_map<kMapBlock, kMapIpt, K_U32_MIX32, true>
                           : (const void*)&dev::k_map<kMapBlock, kMapIpt, K_U32_MIX32, false>;
        case K_F32_POLY3:
            return aligned ? (const void*)&dev::k_map<kMapBlock, kMapIpt, K_F32_POLY3, true>
                           : (const void*)&dev::k_map<kMapBlock, kMapIpt, K_F32_POLY3, false>;
        default:
            return nullptr;
    }
}

// Stack depth 7 holds up to 127 arrays, 11 up to 2047 (kMaxTreeArrays = 1024).
const void* tree_add_kernel_fn(int f32, int aligned, uint32_t k) {
    const bool small = k < 128;
#define SCL_TREE(F, A) (small ? (const void*)&dev::k_tree_add<F, A, 7>   \
                              : (const void*)&dev::k_tree_add<F, A, kTreeLevels>)
    if (f32) return aligned ? SCL_TREE(true, true) : SCL_TREE(true, false);
    return aligned ? SCL_TREE(false, true) : SCL_TREE(false, false);
#undef SCL_TREE
}

const void* large_keyed_kernel_fn(int aligned) {
    return aligned ? (const void*)&dev::k_keyed_large<true> : (const void*)&dev::k_keyed_large<false>;
}

const void* large_keyed_finish_fn() { return (const void*)&dev::k_keyed_large_finish<256>; }

const void* large_scale_fn() { return (const void*)&dev::k_large_scale<256>; }

const void* large_repair_zero_fn() { return (const void*)&dev::k_large_repair_zero<256>; }

}  // namespace scl
