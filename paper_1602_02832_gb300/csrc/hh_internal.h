// Internal declarations shared by the libhh translation units.
#pragma once

#include <cstdint>
#include <string>

#include "../../include/hh.h"

// Sets the process-wide "last error" (used where there is no context) and
// returns code.
int hh_set_global_error(int code, const char *msg);
