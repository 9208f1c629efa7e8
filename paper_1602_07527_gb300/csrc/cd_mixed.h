// Mixed-precision (split-BF16, tcgen05) engine interface.
#pragma once
#include <stddef.h>

namespace cd {
int mixed_init();                                          // CD_OK or a CD_* error
bool mixed_available();                                    // engine built and usable
size_t mixed_workspace_bytes(int n, int nb, int prec);     // extra workspace for mixed calls
}  // namespace cd
