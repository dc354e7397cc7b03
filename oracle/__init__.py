"""CPU oracle for the shaken dynamics -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import anything from here.
The product package never imports it and shares no code with it.
"""
