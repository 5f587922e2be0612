// Internal declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>

namespace ofm {

// Record `fmt` as the calling thread's last error and return `code`.
int fail(int code, const char* fmt, ...);
void clear_error();

}  // namespace ofm
