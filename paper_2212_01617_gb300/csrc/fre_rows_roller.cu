// Row update of the four-roller device (pulled steps; roller nodes stored
// as 0): a translation unit of its own so that these instantiations compile
// alongside the others.
#include "fre_ws.cuh"

namespace fre {

template <int Q, int FMT>
void RollRows<Q, FMT>::update(const Launch &L) {
    WsRowLaunchers<Q, FMT>::template run_roll<WS_UPDATE>(L);
}

template struct RollRows<9, FRE_FP32>;
template struct RollRows<9, FRE_FP16DEV>;
template struct RollRows<9, FRE_BF16DEV>;
template struct RollRows<19, FRE_FP32>;
template struct RollRows<19, FRE_FP16DEV>;
template struct RollRows<19, FRE_BF16DEV>;

}  // namespace fre
