// Definitions of the opaque handle types declared in include/spfhe.h.
#pragma once
#include "internal.h"

struct spfhe_ctx {
    spfhe::Ctx c;
};
struct spfhe_keys {
    spfhe::Keys *k;
};
struct spfhe_ct {
    spfhe::Ct *c;
    bool borrowed = false;   // a graph's result: spfhe_ct_free drops only the handle
};
struct spfhe_pt {
    spfhe::Pt *p;
};
