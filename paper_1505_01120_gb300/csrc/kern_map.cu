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

}  // namespace scl
