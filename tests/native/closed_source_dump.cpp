// Prints the source the closed-tile-pass generator writes for a circuit read
// from standard input ("M amplitude-bytes L delta", then L lines "target mask
// polarity"), after planning the circuit in place with compiled kernels and
// the given changed-bit set, followed by a line "@LAYOUT l k h0 h1 ..." with
// the tile's local-to-address bit order and "@OUT o0 o1 ..." with the tile
// number's bits; with argument "--compile" it also compiles the source with
// NVRTC for sm_103a (no GPU needed) and prints "compiled <bytes>".
#include <cstdio>
#include <cstring>
#include <iostream>
#include <vector>

#include "../../paper_quant_ph_0308158_gb300/csrc/jit.cu"
#include "../../paper_quant_ph_0308158_gb300/csrc/planner.cpp"

namespace qsim {
int num_sms() { return 152; }
void set_last_error(const std::string &) {}
int encode_tile_map(void *, const TilePass &, void *) { return 1; }
}  // namespace qsim

int main(int argc, char **argv)
{
    using namespace qsim;
    uint32_t M = 0;
    int amp = 0;
    size_t L = 0;
    unsigned long long delta = 0;
    if (!(std::cin >> M >> amp >> L >> delta)) return 2;
    std::vector<qsim_step> st(L);
    for (auto &s : st) {
        unsigned long long m = 0, p = 0;
        std::cin >> s.target >> m >> p;
        s.reserved = 0;
        s.ctrl_mask = m;
        s.ctrl_pol = p;
    }
    PlanOptions o;
    o.amp_bytes = (size_t)amp;
    o.strategy = QSIM_STRATEGY_INPLACE;
    o.jit = true;
    o.cancel_adjacent = false;
    o.closed_known = true;
    o.closed_delta = delta;
    Plan plan;
    std::string msg;
    if (make_plan(M, st.data(), L, o, &plan, &msg) != QSIM_OK) {
        std::printf("plan failed: %s\n", msg.c_str());
        return 3;
    }
    if (plan.passes.size() != 1 || !plan.passes[0].tile.closed) {
        std::printf("no closed pass\n");
        return 4;
    }
    const TilePass &t = plan.passes[0].tile;
    const std::string src = generate_closed_source(M, amp, plan.jit_steps.data() + t.jit_off, t.jit_n, t);
    std::cout << src;
    std::cout << "@LAYOUT " << t.l << " " << t.k;
    for (uint32_t q = 0; q < t.nh; ++q) std::cout << " " << t.high[q];
    std::cout << "\n@OUT";
    for (uint32_t q = 0; q < t.nout; ++q) std::cout << " " << t.outpos[q];
    std::cout << "\n";
    if (argc > 1 && std::strcmp(argv[1], "--compile") == 0) {
        Nvrtc &nv = nvrtc();
        if (!nv.ok) {
            std::printf("nvrtc: %s\n", nv.err.c_str());
            return 5;
        }
        nvrtcProgram prog;
        nv.create(&prog, src.c_str(), "closed.cu", 0, nullptr, nullptr);
        const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-default-device"};
        const nvrtcResult r = nv.compile(prog, 3, opts);
        size_t ls = 0;
        nv.log_size(prog, &ls);
        std::string lg(ls, '\0');
        if (ls) nv.log(prog, &lg[0]);
        if (r != NVRTC_SUCCESS) {
            std::printf("compile failed:\n%s\n", lg.c_str());
            return 6;
        }
        size_t cs = 0;
        nv.cubin_size(prog, &cs);
        nv.destroy(&prog);
        std::printf("compiled %zu\n", cs);
    }
    return 0;
}
