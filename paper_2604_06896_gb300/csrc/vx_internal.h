// Internal declarations shared by the host C++ and the CUDA translation units.
#pragma once
#include <cstdint>
#include <string>

#include "../../include/vx.h"

namespace vx {

// Packed target of a half-edge: vertex index in bits 0..27, offx + 1 in
// bits 28..29, offy + 1 in bits 30..31.
constexpr uint32_t TGT_MASK = (1u << 28) - 1;
constexpr int MAX_VERTICES = 1 << 28;

vx_status build_mesh(const double* seeds, int n, double Lx, double Ly, double* vert,
                     int32_t* he, int32_t* face_he, int32_t* edge_id, std::string* err);

void set_error(const std::string& msg);

void seed_order(const double* seeds, int n, double Lx, double Ly, int32_t* order);

}  // namespace vx
