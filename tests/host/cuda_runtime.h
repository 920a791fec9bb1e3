// Empty stand-in for the CUDA runtime header: device code compiled for the host by the
// test harnesses in this directory needs none of its declarations.
#pragma once
