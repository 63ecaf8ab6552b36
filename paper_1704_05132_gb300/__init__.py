"""GB300-native engine for the VNS hot path of Antoniadis & Sifaleras (2017).

Uncapacitated multi-item economic lot-sizing with remanufacturing (ELSR):
best-improvement evaluation of whole VND neighbourhoods over the setup
matrices gM(k,t), gR(k,t), inside VND (Algorithm 1) and GVNS (Algorithm 2),
for single instances, batches, multi-start runs and a serving loop.

The compute path is the C-ABI library ``libelsr.so`` (hand-written sm_103a
CUDA, declared in ``include/elsr.h``); this package only marshals arguments.
The library is loaded on first use and its absence is an error: there is no
CPU fallback.
"""
__all__ = ["gen"]
