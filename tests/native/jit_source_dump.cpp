// Prints the source the compiled-gather generator writes for a circuit read
// from standard input ("M amplitude-bytes L", then L lines "target mask
// polarity"), for tests/test_native_checks.py to evaluate on the host.
#include <cstdio>
#include <iostream>
#include <vector>

#include "../../paper_quant_ph_0308158_gb300/csrc/jit.cu"

namespace qsim {
int num_sms() { return 152; }
void set_last_error(const std::string &) {}
int encode_tile_map(void *, const TilePass &, void *) { return 1; }
}  // namespace qsim

int main()
{
    uint32_t M = 0;
    int amp = 0;
    size_t L = 0;
    if (!(std::cin >> M >> amp >> L)) return 2;
    std::vector<qsim_step> st(L);
    for (auto &s : st) {
        unsigned long long m = 0, p = 0;
        std::cin >> s.target >> m >> p;
        s.reserved = 0;
        s.ctrl_mask = m;
        s.ctrl_pol = p;
    }
    std::cout << qsim::generate_source(M, amp, st.data(), st.size());
    return 0;
}
