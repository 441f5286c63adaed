// Pauli term as the kernels see it (internal; also compiled into run-time
// specialised kernels).
#pragma once

namespace dq {

// One Pauli term in bit space.
struct DevTerm {
    uint64_t f;         // flip mask (bit space)
    uint64_t s;         // sign mask (bit space)
    int32_t nY;         // number of Y factors
    int32_t obs;        // observable index
    double coeff;
};

}  // namespace dq
