// Internal declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>

#include "ofmlmc.h"

// Solver handle: the caller's configuration and its non-dimensional units.
struct ofm_solver {
    ofm_solver_config cfg;
    double p_ref, L, u_ref, t_ref;
};

namespace ofm {

// Record `fmt` as the calling thread's last error and return `code`.
int fail(int code, const char* fmt, ...);
void clear_error();

}  // namespace ofm
