// g g -> t tbar g g, MIXED_BF16 with the separate tensor-core colour pass.
#define RW_STORE_CM CM_STORE_BF16
#define RW_STORE_REGISTER register_gg_ttgg_store_bf16
#include "proc_gg_ttgg_store.cuh"
