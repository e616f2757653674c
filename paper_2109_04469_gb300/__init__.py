"""GB300-native hot path of the explicit electrostatic 1D3V PIC/MCC simulation of a
capacitively coupled RF argon discharge (Vass, Palla & Hartmann, arXiv 2109.04469, §2).

The compute path is hand-written CUDA for sm_103a behind the C-ABI library ``libpic.so``
(header ``include/pic.h``); :mod:`paper_2109_04469_gb300.pic` is its ctypes binding.
Importing this package loads nothing; the binding loads the library on first use and
raises if it has not been built.
"""
